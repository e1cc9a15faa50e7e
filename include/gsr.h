/*
 * gsr.h -- C ABI of the GB300 (sm_103a) Gaussian-splat rasterizer library
 * (libgsr.so): projection, tile binning, forward blend, and the backward blend
 * whose per-splat gradient accumulation is the bottleneck studied by DISTWAR
 * (arXiv 2401.05345).
 *
 * Conventions shared by every entry point
 *  - All pointers are DEVICE pointers unless the argument says "host".  The
 *    caller owns every buffer; the library never allocates device memory.
 *  - Calls are asynchronous on `stream` (a cudaStream_t passed as void*;
 *    NULL = legacy default stream) unless stated otherwise.
 *  - Return value: GSR_OK (0) or a negative status; gsr_status_string() names
 *    it.  Argument errors are detected before anything is launched.  A CUDA
 *    launch or runtime error returns GSR_ECUDA (the CUDA error string is kept
 *    for gsr_last_cuda_error()).  No exception crosses the ABI.
 *  - Gradient outputs ACCUMULATE (+=): the caller zeroes them first
 *    (gsr_preprocess can do that for grad2d in the same pass).
 *  - Images are planar float32 [3][H][W]; per-pixel maps float32/int32 [H][W].
 *  - Alignment: splat2d and grad2d records must start on 16 bytes, tile_ranges
 *    and keys on 8 bytes, binning scratch on 16 bytes (GSR_EINVAL otherwise);
 *    feature arrays may have any 4-byte alignment (16-byte aligned ones are
 *    read with vector loads).
 *  - Tiles: tile_w x tile_h pixels (each a power of two in [8,32], product
 *    <= 512); the grid has gx = ceil(W/tile_w) by gy = ceil(H/tile_h) tiles,
 *    tile id = ty*gx + tx.
 */
#ifndef GSR_H
#define GSR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GSR_OK          0
#define GSR_EINVAL     (-1)  /* bad argument (null pointer, size, option)   */
#define GSR_ECAPACITY  (-2)  /* duplicated keys exceed key_capacity          */
#define GSR_ECUDA      (-3)  /* CUDA runtime / launch error                  */
#define GSR_ETIMEOUT   (-4)  /* reserved: no call waits on the device today   */
#define GSR_ESCRATCH   (-5)  /* scratch buffer smaller than required         */
#define GSR_ELIMIT     (-6)  /* size beyond gsr_bin_sort_static's fixed limit */

typedef void* gsr_stream_t;

/* Pinhole camera.  view: row-major 3x4 [R | t] mapping world to camera
 * coordinates (camera looks down +z, image y down).  A camera-space point
 * (x, y, z) projects to pixel (fx x/z + cx, fy y/z + cy), pixel centres at
 * integer coordinates.  tan_fov*: tangent of the half field of view (the
 * EWA Jacobian clamps x/z to +-1.3 tan_fovx).  campos: world position of the
 * camera, origin of the SH viewing direction.  znear: near-plane cull. */
typedef struct gsr_camera {
    int32_t width, height;
    float view[12];
    float fx, fy, cx, cy;
    float tan_fovx, tan_fovy;
    float campos[3];
    float znear;
} gsr_camera;

/* 2D splat record written by gsr_preprocess, 12 floats (48 bytes) per
 * Gaussian: [0] u [1] v (pixel position), [2] A [3] B [4] C (conic: inverse
 * screen covariance [[A,B],[B,C]]), [5] opacity, [6..8] RGB, [9] depth
 * (camera z), [10..11] zero.  grad2d uses the same stride: [0] dL/du ...
 * [8] dL/db, [9..11] unused (left as the caller initialised them). */
#define GSR_REC 12

/* Reduction tiers of the backward gradient accumulation.
 *  PLAIN   every active pixel-thread issues one atomic add per parameter
 *          (9 per pair) -- the baseline kernel of Sec. III-A, Fig. "Outline
 *          of the gradient computation step".
 *  WARP    every warp that holds at least one active lane reduces the 9
 *          parameters across its 32 lanes in registers (inactive lanes add
 *          zero, Sec. V-A2 / Fig. "modified gradient computation kernel") and
 *          issues one 9-lane red instruction to L2.
 *  HYBRID  balancing threshold (Sec. IV-B, Sec. V-A3): warps with
 *          popc(active) >= threshold reduce at the SM as WARP, the others send
 *          per-lane atomics to the L2 atomic units as PLAIN.
 *  BLOCK   warp partials (or, below the threshold, per-lane values) are
 *          added into the CTA's shared memory; one global red per
 *          (tile, splat, parameter) when the staged batch is retired.
 *  CLUSTER 2 x 2 clusters of tile CTAs: warps at or above the threshold
 *          reduce and add the 9 sums into a hash table spread over the
 *          cluster's distributed shared memory (one owner CTA and slot per
 *          splat id, 1024 slots per CTA; a splat that finds no free slot in
 *          16 probes goes to L2 directly); after a cluster barrier each CTA
 *          issues one global red per (cluster, splat, parameter).  Sparse
 *          warps send per-lane atomics, as in HYBRID.  gsr_backward only
 *          (gsr_backward_batched returns GSR_EINVAL).
 * threshold: 0 = every warp reduces, 33 = none does. */
enum {
    GSR_REDUCE_PLAIN = 0,
    GSR_REDUCE_WARP = 1,
    GSR_REDUCE_HYBRID = 2,
    GSR_REDUCE_BLOCK = 3,
    GSR_REDUCE_CLUSTER = 4
};

/* lane_layout: which pixels of a 16x16 tile share a warp.
 *   0: rows (16 x 2, or 16 x 4 with two pixels per thread),
 *   1: blocks (8 x 4, or 8 x 8 with two pixels per thread). */
typedef struct gsr_backward_opts {
    int32_t reduce_mode;   /* GSR_REDUCE_* */
    int32_t threshold;     /* 0..33, see above */
    int32_t lane_layout;   /* 0 or 1 */
    int32_t store_T;       /* 1: read final_T / n_contrib written by
                              gsr_forward; 0: recompute them in the kernel
                              (final_T / n_contrib may be NULL) */
    int32_t pixels_per_thread; /* 1 (8 warps per tile) or 2 (4 warps; each
                              lane first sums its two pixels' gradients);
                              0 means 1.  PLAIN requires 1. */
    int32_t reserved[3];   /* must be zero */
} gsr_backward_opts;

/* One view of a batched backward (an array of these lives in DEVICE memory).
 * All pointers are device pointers with the meaning and layout they have in
 * gsr_backward; final_T / n_contrib may be NULL when store_T is 0, and so may
 * block_mask (the view's forward block masks, see gsr_forward); 16x16
 * tiles.  splat2d and grad2d must start on 16 bytes (the hybrid tier sends
 * 16-byte vector reds into grad2d); the library cannot check descriptors
 * that live in device memory, so the caller must. */
typedef struct gsr_view {
    int32_t width, height;
    const uint32_t* tile_ranges;
    const uint32_t* point_list;
    const float* splat2d;
    const float* final_T;
    const int32_t* n_contrib;
    const float* dL_dimage;
    float* grad2d;
    const uint8_t* block_mask;
    float bg[3];
    int32_t reserved;
} gsr_view;

/*
 * Cube-map texture workload (the NvDiffRec workload of Sec. VI: learning an
 * environment map from images).  Each pixel with a non-zero direction
 * samples the cube map bilinearly; the backward adds w_k * dL/dout to the
 * gradient of each of the pixel's 4 texels.  The lanes of a warp update
 * different but overlapping texels, the divergent case of Sec. V-A1.
 * Conventions (OpenGL cube maps): face = major axis of the direction (ties:
 * x, then y; positive for components >= 0), faces +x -x +y -y +z -z = 0..5;
 * (sc, tc, ma): +x (-z, -y, |x|), -x (z, -y, |x|), +y (x, z, |y|),
 * -y (x, -z, |y|), +z (x, -y, |z|), -z (-x, -y, |z|); s = (sc/ma + 1)/2,
 * t = (tc/ma + 1)/2; u = s R - 1/2, v = t R - 1/2 evaluated in FP32 with one
 * rounding per operation; taps floor(u) + {0,1} x floor(v) + {0,1} clamped to
 * the face; weights (1-fu)(1-fv), fu(1-fv), (1-fu)fv, fu fv.
 * Layouts: dirs, out, dL_dout [height][width][3] float; tex and grad_tex
 * [6][R][R][4] float (16-byte aligned; channel 3 unused, its gradient stays
 * untouched).  grad_tex accumulates.  6 R^2 < 2^31.
 */
enum {
    GSR_TEX_PLAIN = 0,     /* 3 scalar atomicAdd per tap (the baseline) */
    GSR_TEX_PLAIN_V4 = 1,  /* one red.global.add.v4.f32 per tap */
    GSR_TEX_SERIAL = 2,    /* per tap: lanes on the same texel (match mask) of
                              at least `threshold` lanes are summed by their
                              lowest lane, which pulls each peer in turn and
                              issues one v4 red (SW-S, Sec. V-A1); smaller
                              groups issue per-lane v4 reds */
    GSR_TEX_SORTED = 3,    /* per tap: the warp's (texel, lane) pairs are
                              sorted, summed per run, one v4 red per run */
    GSR_TEX_BLOCK = 4      /* per 16x16-pixel CTA: a 1024-slot shared-memory
                              table (8 probes, then a direct red), flushed
                              with one v4 red per texel at the end */
};
int gsr_cube_forward(int32_t width, int32_t height, const float* dirs, int32_t R, const float* tex,
                     float* out, gsr_stream_t stream);
/* threshold: 0..33, used by GSR_TEX_SERIAL. */
int gsr_cube_backward(int32_t width, int32_t height, const float* dirs, const float* dL_dout, int32_t R,
                      float* grad_tex, int32_t method, int32_t threshold, gsr_stream_t stream);

const char* gsr_status_string(int status);
/* Text of the last CUDA error seen by the library in this thread. */
const char* gsr_last_cuda_error(void);
/* Library ABI version (major*100 + minor). */
int gsr_version(void);

/*
 * Projection ("preprocess") of n 3D Gaussians.  Per Gaussian: camera-space
 * mean, near-plane cull (z <= znear), 3D covariance R(q/|q|) diag(s)^2 R^T,
 * EWA screen covariance J W Sigma W^T J^T + 0.3 I, conic, 3-sigma radius of
 * the larger eigenvalue (eigenvalue discriminant floored at 0.1), tile
 * rectangle (culled when empty), colour max(0, SH(dir) + 0.5) or the given
 * colour.  The paper relies on the 3DGS rasterizer for this step (Sec. VI,
 * "Workloads"; Sec. II-C).
 *   mean [n,3], scale [n,3] (activated, > 0), quat [n,4] (w,x,y,z, any
 *   non-zero norm), opacity [n] (activated, in (0,1)), feat: sh_degree 0..3 ->
 *   SH coefficients [n,(deg+1)^2,3]; sh_degree -1 -> RGB colours [n,3].
 *   cam: host pointer.  Outputs: splat2d [n,GSR_REC] (zeros and radius 0 for
 *   culled Gaussians), radius [n] (int32, 0 = culled).
 *   grad2d_to_zero: optional [n,GSR_REC] buffer zeroed in the same pass.
 */
int gsr_preprocess(int32_t n, int32_t sh_degree, const float* mean, const float* scale,
                   const float* quat, const float* opacity, const float* feat,
                   const gsr_camera* cam, int32_t tile_w, int32_t tile_h, float* splat2d,
                   int32_t* radius, float* grad2d_to_zero, gsr_stream_t stream);

/*
 * Scratch bytes gsr_bin_sort needs for n Gaussians, a W x H image and at
 * most key_capacity duplicated keys (host output *bytes).
 */
int gsr_bin_scratch_bytes(int32_t n, int32_t width, int32_t height, int32_t tile_w,
                          int32_t tile_h, int64_t key_capacity, size_t* bytes);

/*
 * Tile binning: the entries (tile_id << 32 | FP32 bits of depth, Gaussian
 * id) of every (tile, Gaussian) pair in each visible Gaussian's tile
 * rectangle, in the order of a stable sort of the keys emitted in Gaussian
 * order (tile, then depth, then id), and per-tile [start, end) ranges.  This
 * builds the "per-pixel list of primitives" that the gradient computation
 * iterates (Sec. III-A): all pixels of a tile share one depth-sorted list.
 * Computed by hand-written sorts: a stable 3-pass LSD radix sort of the
 * Gaussians' depth keys, then a counting sort that writes each tile's
 * entries in that order (no key array is sorted).
 *   splat2d, radius: from gsr_preprocess.  scratch: scratch_bytes >=
 *   gsr_bin_scratch_bytes().  Outputs: point_list [key_capacity] (Gaussian
 *   ids, first *n_keys valid), tile_ranges [gx*gy*2] (uint32 start, end;
 *   0,0 for empty tiles), keys_out [key_capacity] (optional: sorted keys).
 *   n_keys: HOST pointer, receives the key count.
 * Synchronises `stream` once to read the key count.  Returns GSR_ECAPACITY
 * (with *n_keys set, every tile range empty, nothing else written) when the
 * count exceeds key_capacity: the caller grows the buffers and calls again.
 * A tile grid with 65536 or more tiles per side is GSR_EINVAL.
 */
int gsr_bin_sort(int32_t n, int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                 const float* splat2d, const int32_t* radius, int64_t key_capacity,
                 void* scratch, size_t scratch_bytes, uint32_t* point_list,
                 uint32_t* tile_ranges, uint64_t* keys_out, int64_t* n_keys,
                 gsr_stream_t stream);

/*
 * gsr_bin_sort without the host synchronisation: everything is queued on
 * `stream`, and count_dev (DEVICE pointer, 2 x uint32) receives the key count
 * and a status: 0 ok; 1 more keys than key_capacity (then every tile range
 * is empty and point_list / keys_out are not written, so later kernels of
 * the step see empty lists); 2 inconsistent internal counts (not expected).
 * The caller reads count_dev after the step (e.g. with the loss) and, on
 * status 1, grows the buffers and redoes the step.  Makes the whole step
 * capturable in a CUDA graph.  tile_order: NULL, or DEVICE uint32 [tiles]
 * that receives the longest-first tile order of the new ranges (what
 * gsr_tile_order computes), formed by the last block of the binning's own
 * column scan instead of a launch of its own.  Returns GSR_OK or an
 * argument error.
 */
int gsr_bin_sort_async(int32_t n, int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                       const float* splat2d, const int32_t* radius, int64_t key_capacity,
                       void* scratch, size_t scratch_bytes, uint32_t* point_list,
                       uint32_t* tile_ranges, uint64_t* keys_out, uint32_t* count_dev,
                       uint32_t* tile_order, gsr_stream_t stream);

/*
 * The same binning (same outputs, same arguments and errors) computed with
 * the CUDA Toolkit's CUB radix sorts: the Gaussians sorted by depth, their
 * tile ids emitted in that order, then a stable sort on the tile id.  Kept
 * as the measured comparison for gsr_bin_sort; its scratch size comes from
 * gsr_bin_scratch_bytes_library.
 */
int gsr_bin_scratch_bytes_library(int32_t n, int32_t width, int32_t height, int32_t tile_w,
                                  int32_t tile_h, int64_t key_capacity, size_t* bytes);
int gsr_bin_sort_library(int32_t n, int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                         const float* splat2d, const int32_t* radius, int64_t key_capacity,
                         void* scratch, size_t scratch_bytes, uint32_t* point_list,
                         uint32_t* tile_ranges, uint64_t* keys_out, int64_t* n_keys,
                         gsr_stream_t stream);

/*
 * Allocation-free binning.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory -- code that runs in
 * a process whose GPU memory is owned by another allocator or a fixed
 * budget, and loops that must not pay cudaMalloc's latency and implicit
 * synchronisation.  It computes exactly what gsr_bin_sort computes, but its
 * scratch is a static device array inside libgsr of
 *   (GSR_STATIC_BIN_MAX_GAUSSIANS + 1) * 4 + GSR_STATIC_BIN_MAX_KEYS * 12
 *   + 8 MiB bytes (about 60 MB),
 * reserved on every GPU that loads the library's device code and held until
 * the process exits.  The caller passes only inputs and outputs (as for
 * gsr_bin_sort, plus keys_out, which is required here: it doubles as the
 * sort's alternate key buffer).
 *  - n > GSR_STATIC_BIN_MAX_GAUSSIANS, or a key count above
 *    GSR_STATIC_BIN_MAX_KEYS, returns GSR_ELIMIT (nothing sorted).
 *  - The first call on a device looks up the array's device address (once,
 *    with that device current); make that first call before any stream
 *    capture.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; nothing a call reads from it was left by an earlier call.  Calls
 *    that overlap on the GPU (other streams, other host threads) race on it:
 *    serialise them.
 *  - Synchronises `stream` once (key count), like gsr_bin_sort.
 */
#define GSR_STATIC_BIN_MAX_GAUSSIANS (1 << 20)
#define GSR_STATIC_BIN_MAX_KEYS (1 << 22)
int gsr_bin_sort_static(int32_t n, int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                        const float* splat2d, const int32_t* radius, int64_t key_capacity,
                        uint32_t* point_list, uint32_t* tile_ranges, uint64_t* keys_out,
                        int64_t* n_keys, gsr_stream_t stream);

/*
 * Tile order of the blend kernels: a permutation of the tile ids, longest
 * lists first.  Each tile of a view takes one CTA of the forward and backward
 * kernels, and a CTA's time follows its list length (0 to several thousand
 * entries).  Launching the longest first is the longest-processing-time-first
 * rule of list scheduling; without it the launch ends in a tail of long tiles
 * that started late.  The paper has no counterpart (it launches one thread
 * per pixel and does not discuss scheduling).  Lists are bucketed by length
 * (powers of two, each split in four); tiles of one bucket come in no
 * particular order.  No result depends on the order except the float
 * summation order of the atomic backward tiers, which is not fixed anyway.
 *   tile_ranges: [tiles][2] from binning; order: device uint32 [tiles] (out).
 *   One CTA; asynchronous on `stream`.
 */
int gsr_tile_order(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                   const uint32_t* tile_ranges, uint32_t* order, gsr_stream_t stream);

/*
 * Forward blend: for each pixel, front to back over its tile's list:
 * sigma = A dx^2/2 + B dx dy + C dy^2/2 with (dx,dy) = (u,v) - pixel, skip if
 * sigma < 0; alpha = min(0.99, o exp(-sigma)), skip if alpha < 1/255; stop
 * (excluding this splat) once T (1 - alpha) < 1e-4; C += rgb alpha T;
 * T *= 1 - alpha.  image = C + T bg (Sec. II-C, the forward pass whose
 * per-pixel lists the gradient step walks).
 *   bg: HOST pointer to 3 floats.  Outputs: image [3,H,W]; final_T [H,W]
 *   and n_contrib [H,W] (1-based list position of the last contributor, 0 if
 *   none), both optional (NULL).  tile_order: NULL (tiles in row-major
 *   order) or a permutation of the tile ids from gsr_tile_order, the order
 *   in which CTAs take tiles; ids outside the grid are skipped, and an id
 *   that appears twice is rendered twice (the same values written again).
 *   block_mask: NULL, or device uint8 with one byte per list entry (the
 *   key capacity of the binning) that receives each entry's block mask:
 *   bit b (b = 0..3) is clear only when no pixel of the 8x8 pixel block b
 *   of the entry's tile (b = 2 (y >= 8) + (x >= 8), tile-local pixels) can
 *   reach alpha >= 1/255 with this splat (a conservative test with margins
 *   far above FP32 rounding; bits 4..7 are 0).  Written for every entry the
 *   forward reads: every list position up to the end of the 256-entry batch
 *   in which the tile's last pixel stops.  gsr_backward reads it back.
 */
int gsr_forward(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                const uint32_t* tile_ranges, const uint32_t* point_list, const float* splat2d,
                const float* bg, float* image, float* final_T, int32_t* n_contrib,
                uint8_t* block_mask, const uint32_t* tile_order, gsr_stream_t stream);

/*
 * Forward blend fused with the L1 loss of Sec. II-B (the "loss" stage of the
 * training iteration, Fig. 2): the forward of gsr_forward, and from each
 * composited pixel value `out`, for every channel,
 *   dL_dimage = sign(out - target) (0 where equal),
 *   loss_sum[0] += |out - target|,
 * with the operations of gsr_l1_loss: dL_dimage is bit for bit what
 * gsr_forward followed by gsr_l1_loss writes; the loss is the same float sum
 * added in another order.
 *   target: [3,H,W]; dL_dimage: [3,H,W] (out); loss_sum: device float,
 *   accumulated, or NULL; image: [3,H,W] or NULL (not written).  Other
 *   arguments as gsr_forward.
 */
int gsr_forward_l1(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                   const uint32_t* tile_ranges, const uint32_t* point_list, const float* splat2d,
                   const float* bg, const float* target, float* image, float* final_T, int32_t* n_contrib,
                   float* dL_dimage, float* loss_sum, uint8_t* block_mask, const uint32_t* tile_order,
                   gsr_stream_t stream);

/*
 * Backward blend + per-splat gradient accumulation: the gradient computation
 * step of Sec. III-A.  One thread per pixel walks its tile's list back to
 * front from the pixel's last contributor, recovers T_j = T_{j+1}/(1-alpha_j),
 * and computes for every contributor
 *   dL/drgb = alpha T g,
 *   dL/dalpha = T (rgb.g) - [sum_{k>j} (rgb_k.g) alpha_k T_k + T_final (bg.g)] / (1-alpha),
 *   dL/do = G dL/dalpha, dL/dsigma = -o G dL/dalpha (0 where alpha is capped),
 *   dL/d(A,B,C) = (dx^2/2, dx dy, dy^2/2) dL/dsigma,
 *   dL/d(u,v) = (A dx + B dy, B dx + C dy) dL/dsigma,
 * with g = dL_dimage at the pixel; the 9 values are accumulated into
 * grad2d[id*GSR_REC + 0..8] by the tier in opts (see GSR_REDUCE_*).  Every
 * tier forms the same sum; only the float summation order differs.
 *   final_T, n_contrib: from gsr_forward (ignored when opts->store_T == 0).
 *   bg: HOST pointer.  opts: HOST pointer (NULL = WARP, threshold 0, 16x2,
 *   store_T 1).  tile_order: NULL or a permutation of the tile ids
 *   (gsr_tile_order), as for gsr_forward; it must not repeat an id (a
 *   repeated tile would be accumulated twice).  The cluster tier keeps
 *   row-major order (a cluster is a 2x2 block of neighbouring tiles).
 *   block_mask: NULL, or the block masks that gsr_forward / gsr_forward_l1
 *   wrote for these same lists and splats: each warp then skips the entries
 *   whose bit for its pixel block is clear without recomputing the test.
 *   Read by the configurations whose warps own those 8x8 blocks
 *   (lane_layout 1, pixels_per_thread 2); the others compute the test
 *   themselves.  Masks of other lists or splats give wrong gradients.
 *   grad2d: [n,GSR_REC] starting on 16 bytes (sparse warps of the hybrid
 *   tier add a record's first 8 values with two 16-byte vector reds);
 *   GSR_EINVAL otherwise.
 */
int gsr_backward(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                 const uint32_t* tile_ranges, const uint32_t* point_list,
                 const float* splat2d, const float* bg, const float* final_T,
                 const int32_t* n_contrib, const float* dL_dimage, float* grad2d,
                 const gsr_backward_opts* opts, const uint8_t* block_mask, const uint32_t* tile_order,
                 gsr_stream_t stream);

/*
 * Work order of a batched backward: one item per (view, 16x16 tile), encoded
 * (view << 24) | tile, sorted by decreasing tile-list length (ties keep view
 * then tile order) so the persistent launch schedules the longest tiles first
 * (longest-processing-time order; the paper launches one view at a time).
 *   views: device array [n_views] (n_views <= 256); item_offsets: device
 *   int32 [n_views + 1], exclusive prefix sum of the views' tile counts;
 *   items_out: device uint32 [n_items]; scratch: >= the bytes reported by
 *   gsr_batch_order_scratch_bytes(n_items).  No host synchronisation; sizes are
 *   fixed, so the call can be captured in a CUDA graph.
 */
int gsr_batch_order_scratch_bytes(int32_t n_items, size_t* bytes);
int gsr_batch_order(int32_t n_views, const gsr_view* views, const int32_t* item_offsets, int32_t n_items,
                    void* scratch, size_t scratch_bytes, uint32_t* items_out, gsr_stream_t stream);

/*
 * Batched backward over many views in one persistent launch: CTAs take items
 * (from gsr_batch_order) off one device counter until all are done; each item
 * is the gsr_backward of one tile of one view with the accumulation tier of
 * opts (HOST pointer).  counter: device uint32, reset by this call.
 * ctas_per_sm: CTAs per SM of the persistent grid (0 = the occupancy limit of
 * the chosen kernel).  Asynchronous, no host synchronisation: capturable.
 */
int gsr_backward_batched(int32_t n_views, const gsr_view* views, const uint32_t* items, int32_t n_items,
                         uint32_t* counter, const gsr_backward_opts* opts, int32_t ctas_per_sm,
                         gsr_stream_t stream);

/*
 * Per-Gaussian entry offsets of a binned view, for the deterministic tier:
 * offsets[i] = number of (tile, Gaussian) list entries of Gaussians 0..i-1
 * (exclusive scan of tiles touched, Gaussian order), offsets[n] = key count.
 * The entries of Gaussian i occupy slots offsets[i] .. offsets[i+1]-1 in the
 * row-major order of its tiles.  splat2d / radius as for gsr_bin_sort;
 * offsets: device uint32 [n+1]; scratch >= gsr_entry_offsets_scratch_bytes.
 */
int gsr_entry_offsets_scratch_bytes(int32_t n, size_t* bytes);
int gsr_entry_offsets(int32_t n, int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                      const float* splat2d, const int32_t* radius, void* scratch, size_t scratch_bytes,
                      uint32_t* offsets, gsr_stream_t stream);

/*
 * Deterministic backward: the same gradients as gsr_backward, formed without
 * any float atomic, so the result is bit-identical from run to run whatever
 * else runs on the GPU (the atomic buffering idea of Sec. VIII, "DAB", done
 * in software).  Inside a tile every warp reduces its lanes (fixed shuffle
 * tree) into its own shared-memory slot; the slots are combined in warp
 * order and written to the entry's slot of `partial` (cleared by the call
 * first); a last kernel sums each Gaussian's entries in slot order into
 * grad2d (accumulated).
 *   radius: from gsr_preprocess; entry_offsets: from gsr_entry_offsets (n+1);
 *   partial: device float [partial_entries * 9] scratch.  When
 *   entry_offsets[n] (a device value: the view's entry count) exceeds
 *   partial_entries, no kernel of the call writes anything and grad2d
 *   keeps its values: size partial by the key capacity of the
 *   binning, so that a step whose binning fitted always fits.  Other
 *   arguments (tile_order included) as gsr_backward.  opts: lane_layout,
 *   store_T, pixels_per_thread are used (reduce_mode and threshold are
 *   ignored: every active warp reduces).  The
 *   bits of the result depend on lane_layout and pixels_per_thread (they fix
 *   the summation order), not on scheduling, nor on whether block_mask (as
 *   for gsr_backward) is given.
 */
int gsr_backward_deterministic(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                               const uint32_t* tile_ranges, const uint32_t* point_list,
                               const float* splat2d, const int32_t* radius, int32_t n,
                               const uint32_t* entry_offsets, const float* bg, const float* final_T,
                               const int32_t* n_contrib, const float* dL_dimage, float* partial,
                               int64_t partial_entries, float* grad2d, const gsr_backward_opts* opts,
                               const uint8_t* block_mask, const uint32_t* tile_order, gsr_stream_t stream);

/*
 * Traversal statistics of gsr_backward (nothing else is written): walks the
 * same lists as the backward with the same skip tests and fills the
 * device array hist[38] (uint64, zeroed first):
 *   hist[k], k = 0..32: number of (warp, splat) steps with k active lanes --
 *     the active-threads-per-warp histogram of Sec. III-B, Observation 2;
 *   hist[33]: active (pixel, splat) pairs (each adds 9 gradient values);
 *   hist[34]: examined pairs (sum of n_contrib);
 *   hist[35]: warp steps taken;
 *   hist[36]: warp steps that pass the kernels' per-warp footprint cull;
 *   hist[37]: of those, steps with no active lane.
 * lane_layout as in gsr_backward_opts.  n_contrib from gsr_forward.
 */
int gsr_backward_stats(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                       const uint32_t* tile_ranges, const uint32_t* point_list,
                       const float* splat2d, const int32_t* n_contrib, int32_t lane_layout,
                       uint64_t* hist, gsr_stream_t stream);

/*
 * Global red counts of one backward launch: the traversal of gsr_backward
 * with the tier and threshold of opts (PLAIN, WARP or HYBRID; store_T = 1),
 * every global red replaced by counting it, nothing else written.  Gives the
 * L2 atomic traffic of a tier (Sec. III-A: the atomic operations per
 * iteration; Sec. IV-B: the balancing threshold moves warps between the SM
 * and the L2).  counts: device uint64 [39], overwritten:
 *   [0] scalar red warp instructions, [1] red.v4 warp instructions,
 *   [2] floats added at the L2, [3] lane-level red operations (the requests
 *   before any coalescing), [4] (warp, splat) steps walked, [5] of those
 *   with at least one active lane, [6 + a] steps with exactly a active
 *   lanes, a = 0..32 (the per-warp activity of Sec. III-B, Fig. 5, for
 *   this configuration).
 * Other arguments as gsr_backward (no upstream gradient or grad2d needed).
 */
int gsr_backward_red_counts(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                            const uint32_t* tile_ranges, const uint32_t* point_list, const float* splat2d,
                            const float* final_T, const int32_t* n_contrib, const gsr_backward_opts* opts,
                            const uint8_t* block_mask, const uint32_t* tile_order, uint64_t* counts,
                            gsr_stream_t stream);

/*
 * Backward projection: chain rule from grad2d to the 3D parameters through
 * the conic inverse, the EWA Jacobian (exact derivative, zero through an
 * active frustum clamp), the covariance R S S^T R^T, the quaternion
 * normalisation and the SH basis (zero on channels clamped at 0).  The paper
 * only states that gradients of all parameters are computed (Sec. II-C).
 * Inputs as gsr_preprocess plus radius and grad2d [n,GSR_REC].  Outputs
 * ACCUMULATE: dmean [n,3], dscale [n,3], dquat [n,4], dopacity [n], dfeat
 * (layout of feat).  Gaussians with radius 0 are left untouched.
 */
int gsr_backward_project(int32_t n, int32_t sh_degree, const float* mean, const float* scale,
                         const float* quat, const float* opacity, const float* feat,
                         const gsr_camera* cam, const int32_t* radius, const float* grad2d,
                         float* dmean, float* dscale, float* dquat, float* dopacity,
                         float* dfeat, gsr_stream_t stream);
/*
 * The same, but the outputs are written instead of accumulated: every
 * element of every Gaussian's gradients is stored (zero for Gaussians with
 * radius 0), so a single-view step needs neither a zero fill nor a read of
 * the previous values.
 */
int gsr_backward_project_store(int32_t n, int32_t sh_degree, const float* mean, const float* scale,
                               const float* quat, const float* opacity, const float* feat,
                               const gsr_camera* cam, const int32_t* radius, const float* grad2d,
                               float* dmean, float* dscale, float* dquat, float* dopacity,
                               float* dfeat, gsr_stream_t stream);

/*
 * L1 photometric loss of Sec. II-B (difference to the reference image):
 * dL_dimage[i] = sign(image[i] - target[i]) (0 where equal) and, if loss_sum
 * is not NULL, loss_sum[0] += sum |image - target| (device float).
 */
int gsr_l1_loss(int64_t count, const float* image, const float* target, float* dL_dimage,
                float* loss_sum, gsr_stream_t stream);

/*
 * Parameter activations of the trainable scene (the 3DGS parameterisation the
 * paper's workload trains, Sec. VI): scale = exp(log_scale) [n,3],
 * opacity = 1 / (1 + exp(-opacity_logit)) [n].
 * gsr_activate_backward ACCUMULATES dL/dlog_scale += dL/dscale * scale and
 * dL/dlogit += dL/dopacity * o (1 - o), from the activated values.
 */
int gsr_activate(int64_t n, const float* log_scale, const float* opacity_logit, float* scale,
                 float* opacity, gsr_stream_t stream);
int gsr_activate_backward(int64_t n, const float* scale, const float* opacity, const float* dscale,
                          const float* dopacity, float* dlog_scale, float* dopacity_logit,
                          gsr_stream_t stream);

/*
 * Adam (Kingma & Ba) on a flat float array of n parameters, step >= 1:
 * m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).
 * The optimizer step of the training loop (Sec. II-B, Fig. 2).
 */
int gsr_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr,
                  float beta1, float beta2, float eps, int32_t step, gsr_stream_t stream);

/*
 * Scatter-add of n records of 9 floats: out[idx[i]*stride + q] += vals[9*i + q]
 * (q = 0..8) -- the gradient accumulation with arbitrary destinations, where
 * the lanes of a warp may update different primitives.  method:
 *   0 PLAIN  one atomic add per value (the baseline of Sec. III-A);
 *   1 SERIAL the serialized warp reduction of Sec. V-A1 (SW-S): lanes with
 *            equal destinations are grouped (match_any); groups of at least
 *            `threshold` lanes are summed by their lowest lane, which pulls
 *            the 9 values of each peer in turn and issues one red per value;
 *            smaller groups use per-lane atomics;
 *   2 SORTED the warp's destinations are sorted in registers (bitonic
 *            network) and a segmented shuffle scan sums each run of equal
 *            destinations, whose last lane issues one red per value
 *            (threshold ignored).
 * idx [n] (uint32 row indices), vals [n,9], out [rows,stride] (stride >= 9,
 * accumulated).  Every method forms the same sums; only the float summation
 * order differs.  When stride is a multiple of 4 and out is 16-byte aligned,
 * methods 1 and 2 send a record's 9 values as two 4-wide vector reds and one
 * scalar red.
 */
int gsr_scatter_add9(int64_t n, const uint32_t* idx, const float* vals, float* out, int32_t stride,
                     int32_t method, int32_t threshold, gsr_stream_t stream);

/*
 * Microbenchmark of the L2 atomic (red) path, the roofline of the atomic
 * accumulation (Sec. II-A, Sec. III-A: atomics are processed by the atomic
 * units at the L2 slices).  Each pattern is one way warps send adds:
 *   0: every lane adds 1 float to its own address (coalesced, distinct);
 *   1: all 32 lanes of a warp add to one address (contended);
 *   2: 9 lanes of a warp add to the 9 floats of one 48-byte record (the
 *      reduced tiers' one red per dense warp step);
 *   3: every lane adds the same record's 9 floats (the PLAIN tier's warp
 *      with all lanes active);
 *   4: every lane adds 4 floats to its own 16-byte slot (red.v4, distinct);
 *   5: every lane sends two red.v4 and one scalar red to one record per warp
 *      (the hybrid tier's sparse warp with all lanes active);
 *   6: every lane adds 9 floats to its own record (PLAIN without contention).
 * active_lanes (1..32): in the patterns with one address or record per warp
 * (1, 3, 5) only lanes 0..active_lanes-1 send (a warp step with that many
 * active pixels); the other patterns use every lane.
 * Issues `iters` rounds over a grid of `blocks` x 256 threads; buffer holds
 * buffer_floats floats (device, 16-byte aligned, accumulated into).  Floats
 * added are reported in *adds (host).
 */
int gsr_bench_red(int32_t pattern, int32_t active_lanes, int32_t blocks, int32_t iters, float* buffer,
                  int64_t buffer_floats, int64_t* adds, gsr_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GSR_H */
