// Forward blend, backward blend + per-splat gradient accumulation, and the
// traversal statistics, for one view (kernels in raster_common.cuh).
#include "raster_common.cuh"

#ifndef GSR_FORWARD_PPT
#define GSR_FORWARD_PPT 2
#endif

namespace gsr {
namespace {

// One CTA: the longest-first tile order (tile_order_block).
__global__ void __launch_bounds__(kOrderThreads)
tile_order_kernel(int tiles, const uint2* __restrict__ ranges, uint32_t* __restrict__ order) {
    __shared__ uint32_t cnt[kOrderBuckets];
    tile_order_block(tiles, ranges, order, cnt);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// L1: the epilogue also forms the L1 loss of each pixel (target, dL_dimage,
// loss_sum; image may then be NULL).
template <class SH, bool L1>
__global__ void __launch_bounds__(SH::NT)
forward_kernel(RasterGeom g, const uint2* __restrict__ ranges, const uint32_t* __restrict__ point_list,
               const float* __restrict__ splat2d, float bg0, float bg1, float bg2, float* __restrict__ image,
               float* __restrict__ final_T, int* __restrict__ n_contrib, const uint32_t* __restrict__ order,
               const float* __restrict__ target, float* __restrict__ dimg, float* __restrict__ loss_sum,
               uint8_t* __restrict__ block_mask) {
    constexpr int PPT = SH::B / SH::NT;
    __shared__ float4 s_a[SH::B];
    __shared__ float4 s_b[SH::B];
    __shared__ float s_c[SH::B];
    __shared__ unsigned s_mask[SH::B];
    const int tile = order ? (int)order[blockIdx.x] : (int)blockIdx.x;
    if ((unsigned)tile >= (unsigned)(g.gx * g.gy)) return;  // not a tile id
    const int ox = (tile % g.gx) * SH::TWd, oy = (tile / g.gx) * SH::THd;
    float px[PPT], py[PPT], T[PPT], C[PPT][3];
    bool inside[PPT];
    int last[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        int lx, ly;
        SH::pixel(threadIdx.x, q, lx, ly);
        px[q] = (float)(ox + lx);
        py[q] = (float)(oy + ly);
        inside[q] = ox + lx < g.W && oy + ly < g.H;
    }
    walk_front<SH, true>(ranges[tile], point_list, splat2d, px, py, inside, ox, oy, s_a, s_b, s_c, s_mask, T, last,
                         C, nullptr, block_mask);
    const size_t HW = (size_t)g.W * g.H;
    float labs = 0.0f;  // L1: sum of |out - target| over this thread's pixels
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        if (!inside[q]) continue;
        const size_t pix = (size_t)py[q] * g.W + (size_t)px[q];
        const float out[3] = {__fmaf_rn(T[q], bg0, C[q][0]), __fmaf_rn(T[q], bg1, C[q][1]),
                              __fmaf_rn(T[q], bg2, C[q][2])};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            if (!L1 || image) image[ch * HW + pix] = out[ch];
            if (L1) {  // the operations of gsr_l1_loss
                const float d = __fsub_rn(out[ch], target[ch * HW + pix]);
                dimg[ch * HW + pix] = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
                labs += fabsf(d);
            }
        }
        if (final_T) final_T[pix] = T[q];
        if (n_contrib) n_contrib[pix] = last[q];
    }
    if (L1 && loss_sum) {
        __shared__ float s_l[SH::NW];
        labs = warp_sum(labs);
        if ((threadIdx.x & 31) == 0) s_l[threadIdx.x >> 5] = labs;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.0f;
#pragma unroll
            for (int w = 0; w < SH::NW; ++w) t += s_l[w];
            atomicAdd(loss_sum, t);
        }
    }
}

template <class SH, int MODE, bool STORE_T>
__global__ void __launch_bounds__(SH::NT)
backward_kernel(BwdArgs p) {
    __shared__ BwdSmem<SH::B, MODE> sm;
    const int tile = p.order ? (int)p.order[blockIdx.x] : (int)blockIdx.x;
    if ((unsigned)tile >= (unsigned)(p.g.gx * p.g.gy)) return;  // not a tile id
    backward_tile<SH, MODE, STORE_T>(p, tile, sm);
}

// Cluster tier: tiles (blockIdx.x, blockIdx.y) in 2 x 2 clusters (the grid is
// rounded up to even sizes; CTAs past the image only take part in the
// cluster's two barriers and its table).  Dynamic shared memory: key[cap],
// val[cap][9] of this CTA's part of the cluster table.
template <class SH, bool STORE_T>
__global__ void __cluster_dims__(2, 2, 1) __launch_bounds__(SH::NT)
backward_cluster_kernel(BwdArgs p, int cap) {
    __shared__ BwdSmem<SH::B, kModeCluster> sm;
    extern __shared__ uint32_t s_tab[];
    uint32_t* key = s_tab;
    float* val = reinterpret_cast<float*>(s_tab + cap);
    for (int i = threadIdx.x; i < cap; i += SH::NT) key[i] = kSlotEmpty;
    for (int i = threadIdx.x; i < cap * 9; i += SH::NT) val[i] = 0.0f;
    ClusterTab ct;
    ct.cap = cap;
    ct.key_base = (uint32_t)__cvta_generic_to_shared(key);
    ct.val_base = (uint32_t)__cvta_generic_to_shared(val);
    cluster_sync_all();  // every part of the table is initialised
    const int tx = blockIdx.x, ty = blockIdx.y;
    if (tx < p.g.gx && ty < p.g.gy) backward_tile<SH, kModeCluster, STORE_T>(p, ty * p.g.gx + tx, sm, DetSmem{}, &ct);
    cluster_sync_all();  // every remote add into this CTA's part has landed
    for (int i = threadIdx.x; i < cap * 9; i += SH::NT) {
        const uint32_t id = key[i / 9];
        const float v = val[i];
        if (id != kSlotEmpty && v != 0.0f) red_add(p.grad2d + (size_t)id * GSR_REC + (i % 9), v);
    }
}

// Counts of the backward traversal (no gradients written): per (warp, splat)
// step the number of active lanes -> hist[0..32]; hist[33] = active pairs,
// hist[34] = examined pairs (sum of n_contrib), hist[35] = warp steps with at
// least one lane still walking, hist[36] = those steps that pass the per-warp
// footprint cull, hist[37] = culled-in steps without any active lane.  The
// histogram is the active-lanes-per-warp measurement of Sec. III-B
// (Observation 2).  One pixel per thread.
template <class SH>
__global__ void __launch_bounds__(SH::NT)
stats_kernel(BwdArgs p, unsigned long long* __restrict__ hist) {
    constexpr int B = SH::B;
    __shared__ float4 s_a[B];
    __shared__ float4 s_b[B];
    __shared__ unsigned long long s_h[38];
    __shared__ unsigned s_mask[B];
    __shared__ int s_maxlast;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    const int ox = (tile % p.g.gx) * SH::TWd, oy = (tile / p.g.gx) * SH::THd;
    int lx, ly;
    SH::pixel(tid, 0, lx, ly);
    const int px = ox + lx, py = oy + ly;
    const bool inside = px < p.g.W && py < p.g.H;
    const uint2 rg = p.ranges[tile];
    const int nlist = (int)(rg.y - rg.x);
    const size_t pix = (size_t)py * p.g.W + px;
    const int last = inside ? min(max(p.n_contrib[pix], 0), nlist) : 0;
    for (int i = tid; i < 38; i += B) s_h[i] = 0ull;
    if (tid == 0) s_maxlast = 0;
    __syncthreads();
    const int wlast = __reduce_max_sync(kFull, last);
    if (lane == 0) atomicMax(&s_maxlast, wlast);
    atomicAdd(&s_h[34], (unsigned long long)last);
    __syncthreads();
    const int maxlast = s_maxlast;
    unsigned long long active_pairs = 0;
    for (int top = maxlast; top > 0; top -= B) {
        const int cnt = min(B, top);
        __syncthreads();
        stage_batch<SH, false, false>(cnt, [&](int e) { return rg.x + (uint32_t)(top - 1 - e); }, p.point_list,
                                      p.splat2d, ox, oy, s_a, s_b, nullptr, nullptr, s_mask, nullptr, nullptr);
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const int pos = top - 1 - k;
            if (pos >= wlast) continue;
            const float4 a = s_a[k], b = s_b[k];
            SplatEval e;
            const bool active = (pos < last) && eval_splat(a.x, a.y, a.z, a.w, b.x, b.y, (float)px, (float)py, e);
            const unsigned m = __ballot_sync(kFull, active);
            active_pairs += active ? 1ull : 0ull;
            if (lane == 0) {
                atomicAdd(&s_h[__popc(m)], 1ull);
                atomicAdd(&s_h[35], 1ull);
                if ((s_mask[k] >> warp) & 1u) {
                    atomicAdd(&s_h[36], 1ull);
                    if (m == 0u) atomicAdd(&s_h[37], 1ull);
                }
            }
        }
    }
    atomicAdd(&s_h[33], active_pairs);
    __syncthreads();
    for (int i = tid; i < 38; i += B)
        if (s_h[i]) atomicAdd(&hist[i], s_h[i]);
}

template <class SH, bool STORE_T>
__global__ void __launch_bounds__(SH::NT)
backward_det_kernel(BwdArgs p) {
    __shared__ BwdSmem<SH::B, kModeDet> sm;
    if (p.entry_off[p.n] > p.partial_cap) return;  // partial too small: nothing is written
    const int tile = p.order ? (int)p.order[blockIdx.x] : (int)blockIdx.x;
    if ((unsigned)tile >= (unsigned)(p.g.gx * p.g.gy)) return;  // not a tile id
    extern __shared__ float s_dyn[];
    DetSmem det;
    det.part = s_dyn;
    det.wflags = reinterpret_cast<unsigned*>(s_dyn + SH::NW * kDetGroup * 9);
    backward_tile<SH, kModeDet, STORE_T>(p, tile, sm, det);
}

// Clears the 9 slots of every entry (nothing when the entry count exceeds cap).
__global__ void zero_partial_kernel(int n, const uint32_t* __restrict__ off, uint32_t cap,
                                    float* __restrict__ partial) {
    const uint32_t cnt = off[n];
    if (cnt > cap) return;
    const size_t total = 9 * (size_t)cnt;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x)
        partial[i] = 0.0f;
}

// grad2d[i] += sum of Gaussian i's entry partials, in slot (tile) order.
__global__ void entries_reduce_kernel(int n, const uint32_t* __restrict__ off, const float* __restrict__ partial,
                                      uint32_t cap, float* __restrict__ grad2d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || off[n] > cap) return;
    const uint32_t e0 = off[i], e1 = off[i + 1];
    if (e0 == e1) return;
    float acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = 0.0f;
    for (uint32_t e = e0; e < e1; ++e)
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] += partial[9 * (size_t)e + q];
    float* rec = grad2d + (size_t)i * GSR_REC;
#pragma unroll
    for (int q = 0; q < 9; ++q) rec[q] += acc[q];
}

template <class SH, bool STORE_T>
int launch_det(int tiles, const BwdArgs& a, cudaStream_t s) {
    constexpr size_t dyn = sizeof(float) * SH::NW * kDetGroup * 9 + sizeof(uint32_t) * SH::B;
    auto k = backward_det_kernel<SH, STORE_T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return cuda_fail(e);
    k<<<tiles, SH::NT, dyn, s>>>(a);
    return check_launch();
}

template <int LAYOUT, int PPT>
int launch_det_store(bool store, int tiles, const BwdArgs& a, cudaStream_t s) {
    using SH = Shape<16, 16, LAYOUT, PPT>;
    return store ? launch_det<SH, true>(tiles, a, s) : launch_det<SH, false>(tiles, a, s);
}

template <int MODE, int LAYOUT, int PPT, bool STORE_T>
void launch_bwd(int tiles, const BwdArgs& a, cudaStream_t s) {
    using SH = Shape<16, 16, LAYOUT, PPT>;
    backward_kernel<SH, MODE, STORE_T><<<tiles, SH::NT, 0, s>>>(a);
}

template <int MODE, int PPT>
void launch_bwd_lay(int layout, bool store, int tiles, const BwdArgs& a, cudaStream_t s) {
    if (layout == 0) {
        if (store) launch_bwd<MODE, 0, PPT, true>(tiles, a, s);
        else launch_bwd<MODE, 0, PPT, false>(tiles, a, s);
    } else {
        if (store) launch_bwd<MODE, 1, PPT, true>(tiles, a, s);
        else launch_bwd<MODE, 1, PPT, false>(tiles, a, s);
    }
}

// Cluster-table slots per CTA (40 bytes each).
constexpr int kClusterSlots = 1024;

template <int LAYOUT, int PPT, bool STORE_T>
int launch_cluster(const BwdArgs& a, cudaStream_t s) {
    using SH = Shape<16, 16, LAYOUT, PPT>;
    constexpr size_t dyn = (size_t)kClusterSlots * 10 * sizeof(uint32_t);
    auto k = backward_cluster_kernel<SH, STORE_T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return cuda_fail(e);
    const dim3 grid((unsigned)((a.g.gx + 1) / 2 * 2), (unsigned)((a.g.gy + 1) / 2 * 2));
    k<<<grid, SH::NT, dyn, s>>>(a, kClusterSlots);
    return check_launch();
}

template <int LAYOUT, int PPT>
int launch_cluster_store(bool store, const BwdArgs& a, cudaStream_t s) {
    return store ? launch_cluster<LAYOUT, PPT, true>(a, s) : launch_cluster<LAYOUT, PPT, false>(a, s);
}

template <int MODE>
void launch_bwd_mode(int ppt, int layout, bool store, int tiles, const BwdArgs& a, cudaStream_t s) {
    if (ppt == 2) launch_bwd_lay<MODE, 2>(layout, store, tiles, a, s);
    else launch_bwd_lay<MODE, 1>(layout, store, tiles, a, s);
}

}  // namespace

// Options check shared with the batched entry point.
int check_bwd_opts(const gsr_backward_opts& o) {
    if (o.reduce_mode < GSR_REDUCE_PLAIN || o.reduce_mode > GSR_REDUCE_CLUSTER) return GSR_EINVAL;
    if (o.threshold < 0 || o.threshold > 33 || (o.lane_layout != 0 && o.lane_layout != 1)) return GSR_EINVAL;
    if (o.store_T != 0 && o.store_T != 1) return GSR_EINVAL;
    if (o.pixels_per_thread < 0 || o.pixels_per_thread > 2) return GSR_EINVAL;
    if (o.reduce_mode == GSR_REDUCE_PLAIN && o.pixels_per_thread == 2) return GSR_EINVAL;
    for (int i = 0; i < 3; ++i)
        if (o.reserved[i] != 0) return GSR_EINVAL;
    return GSR_OK;
}

}  // namespace gsr

using namespace gsr;

extern "C" int gsr_tile_order(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                              const uint32_t* tile_ranges, uint32_t* order, gsr_stream_t stream) {
    if (width <= 0 || height <= 0 || !tile_ranges || !order) return GSR_EINVAL;
    if (tile_w != 16 || tile_h != 16 || !aligned8(tile_ranges)) return GSR_EINVAL;
    const int tiles = ((width + 15) / 16) * ((height + 15) / 16);
    tile_order_kernel<<<1, kOrderThreads, 0, (cudaStream_t)stream>>>(tiles, reinterpret_cast<const uint2*>(tile_ranges),
                                                                     order);
    return check_launch();
}

extern "C" int gsr_forward(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                           const uint32_t* tile_ranges, const uint32_t* point_list, const float* splat2d,
                           const float* bg, float* image, float* final_T, int32_t* n_contrib,
                           uint8_t* block_mask, const uint32_t* tile_order, gsr_stream_t stream) {
    if (width <= 0 || height <= 0 || !tile_ranges || !splat2d || !bg || !image) return GSR_EINVAL;
    if (!aligned16(splat2d) || !aligned8(tile_ranges)) return GSR_EINVAL;
    if (tile_w != 16 || tile_h != 16) return GSR_EINVAL;
    RasterGeom g{width, height, (width + 15) / 16, (height + 15) / 16};
    using SH = Shape<16, 16, 1, GSR_FORWARD_PPT>;
    forward_kernel<SH, false><<<g.gx * g.gy, SH::NT, 0, (cudaStream_t)stream>>>(
        g, reinterpret_cast<const uint2*>(tile_ranges), point_list, splat2d, bg[0], bg[1], bg[2], image, final_T,
        n_contrib, tile_order, nullptr, nullptr, nullptr, block_mask);
    return check_launch();
}

extern "C" int gsr_forward_l1(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                              const uint32_t* tile_ranges, const uint32_t* point_list, const float* splat2d,
                              const float* bg, const float* target, float* image, float* final_T,
                              int32_t* n_contrib, float* dL_dimage, float* loss_sum, uint8_t* block_mask,
                              const uint32_t* tile_order, gsr_stream_t stream) {
    if (width <= 0 || height <= 0 || !tile_ranges || !splat2d || !bg || !target || !dL_dimage) return GSR_EINVAL;
    if (!aligned16(splat2d) || !aligned8(tile_ranges)) return GSR_EINVAL;
    if (tile_w != 16 || tile_h != 16) return GSR_EINVAL;
    RasterGeom g{width, height, (width + 15) / 16, (height + 15) / 16};
    using SH = Shape<16, 16, 1, GSR_FORWARD_PPT>;
    forward_kernel<SH, true><<<g.gx * g.gy, SH::NT, 0, (cudaStream_t)stream>>>(
        g, reinterpret_cast<const uint2*>(tile_ranges), point_list, splat2d, bg[0], bg[1], bg[2], image, final_T,
        n_contrib, tile_order, target, dL_dimage, loss_sum, block_mask);
    return check_launch();
}

extern "C" int gsr_backward(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                            const uint32_t* tile_ranges, const uint32_t* point_list, const float* splat2d,
                            const float* bg, const float* final_T, const int32_t* n_contrib,
                            const float* dL_dimage, float* grad2d, const gsr_backward_opts* opts,
                            const uint8_t* block_mask, const uint32_t* tile_order, gsr_stream_t stream_) {
    gsr_backward_opts o = {GSR_REDUCE_WARP, 0, 0, 1, 1, {0, 0, 0}};
    if (opts) o = *opts;
    if (width <= 0 || height <= 0 || !tile_ranges || !splat2d || !bg || !dL_dimage || !grad2d) return GSR_EINVAL;
    // grad2d records take 16-byte vector reds (sparse warps of the hybrid tier)
    if (!aligned16(splat2d) || !aligned16(grad2d) || !aligned8(tile_ranges)) return GSR_EINVAL;
    if (tile_w != 16 || tile_h != 16) return GSR_EINVAL;
    if (check_bwd_opts(o) != GSR_OK) return GSR_EINVAL;
    if (o.store_T && (!final_T || !n_contrib)) return GSR_EINVAL;
    BwdArgs a = {};
    a.g = RasterGeom{width, height, (width + 15) / 16, (height + 15) / 16};
    a.ranges = reinterpret_cast<const uint2*>(tile_ranges);
    a.point_list = point_list;
    a.splat2d = splat2d;
    a.bg0 = bg[0]; a.bg1 = bg[1]; a.bg2 = bg[2];
    a.final_T = final_T;
    a.n_contrib = n_contrib;
    a.dL_dimage = dL_dimage;
    a.grad2d = grad2d;
    a.threshold = o.threshold;
    a.order = tile_order;
    a.block_mask = block_mask;
    const int tiles = a.g.gx * a.g.gy;
    cudaStream_t s = (cudaStream_t)stream_;
    const bool st = o.store_T != 0;
    const int ppt = o.pixels_per_thread == 2 ? 2 : 1;
    switch (o.reduce_mode) {
        case GSR_REDUCE_PLAIN: launch_bwd_lay<GSR_REDUCE_PLAIN, 1>(o.lane_layout, st, tiles, a, s); break;
        case GSR_REDUCE_WARP: launch_bwd_mode<GSR_REDUCE_WARP>(ppt, o.lane_layout, st, tiles, a, s); break;
        case GSR_REDUCE_HYBRID: launch_bwd_mode<GSR_REDUCE_HYBRID>(ppt, o.lane_layout, st, tiles, a, s); break;
        case GSR_REDUCE_BLOCK: launch_bwd_mode<GSR_REDUCE_BLOCK>(ppt, o.lane_layout, st, tiles, a, s); break;
        default:
            if (ppt == 2) return o.lane_layout ? launch_cluster_store<1, 2>(st, a, s) : launch_cluster_store<0, 2>(st, a, s);
            return o.lane_layout ? launch_cluster_store<1, 1>(st, a, s) : launch_cluster_store<0, 1>(st, a, s);
    }
    return check_launch();
}

extern "C" int gsr_backward_stats(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                                  const uint32_t* tile_ranges, const uint32_t* point_list,
                                  const float* splat2d, const int32_t* n_contrib, int32_t lane_layout,
                                  uint64_t* hist, gsr_stream_t stream) {
    if (width <= 0 || height <= 0 || !tile_ranges || !splat2d || !n_contrib || !hist) return GSR_EINVAL;
    if (!aligned16(splat2d) || !aligned8(tile_ranges)) return GSR_EINVAL;
    if (tile_w != 16 || tile_h != 16 || (lane_layout != 0 && lane_layout != 1)) return GSR_EINVAL;
    BwdArgs a = {};
    a.g = RasterGeom{width, height, (width + 15) / 16, (height + 15) / 16};
    a.ranges = reinterpret_cast<const uint2*>(tile_ranges);
    a.point_list = point_list;
    a.splat2d = splat2d;
    a.n_contrib = n_contrib;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(hist, 0, 38 * sizeof(uint64_t), s);
    if (e != cudaSuccess) return cuda_fail(e);
    const int tiles = a.g.gx * a.g.gy;
    if (lane_layout == 0) stats_kernel<Shape<16, 16, 0, 1>><<<tiles, 256, 0, s>>>(a, (unsigned long long*)hist);
    else stats_kernel<Shape<16, 16, 1, 1>><<<tiles, 256, 0, s>>>(a, (unsigned long long*)hist);
    return check_launch();
}

extern "C" int gsr_backward_red_counts(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                                       const uint32_t* tile_ranges, const uint32_t* point_list,
                                       const float* splat2d, const float* final_T, const int32_t* n_contrib,
                                       const gsr_backward_opts* opts, const uint8_t* block_mask,
                                       const uint32_t* tile_order, uint64_t* counts, gsr_stream_t stream_) {
    if (width <= 0 || height <= 0 || !tile_ranges || !splat2d || !final_T || !n_contrib || !opts || !counts)
        return GSR_EINVAL;
    if (!aligned16(splat2d) || !aligned8(tile_ranges) || !aligned8(counts)) return GSR_EINVAL;
    if (tile_w != 16 || tile_h != 16) return GSR_EINVAL;
    const gsr_backward_opts o = *opts;
    if (check_bwd_opts(o) != GSR_OK || !o.store_T) return GSR_EINVAL;
    if (o.reduce_mode != GSR_REDUCE_PLAIN && o.reduce_mode != GSR_REDUCE_WARP && o.reduce_mode != GSR_REDUCE_HYBRID)
        return GSR_EINVAL;
    BwdArgs a = {};
    a.g = RasterGeom{width, height, (width + 15) / 16, (height + 15) / 16};
    a.ranges = reinterpret_cast<const uint2*>(tile_ranges);
    a.point_list = point_list;
    a.splat2d = splat2d;
    a.final_T = final_T;
    a.n_contrib = n_contrib;
    a.threshold = o.threshold;
    a.order = tile_order;
    a.block_mask = block_mask;
    a.counts = reinterpret_cast<unsigned long long*>(counts);
    a.count_tier = o.reduce_mode;
    cudaStream_t s = (cudaStream_t)stream_;
    cudaError_t e = cudaMemsetAsync(counts, 0, kCountSlots * sizeof(uint64_t), s);
    if (e != cudaSuccess) return cuda_fail(e);
    launch_bwd_mode<kModeCount>(o.pixels_per_thread == 2 ? 2 : 1, o.lane_layout, true, a.g.gx * a.g.gy, a, s);
    return check_launch();
}

extern "C" int gsr_backward_deterministic(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                                          const uint32_t* tile_ranges, const uint32_t* point_list,
                                          const float* splat2d, const int32_t* radius, int32_t n,
                                          const uint32_t* entry_offsets, const float* bg, const float* final_T,
                                          const int32_t* n_contrib, const float* dL_dimage, float* partial,
                                          int64_t partial_entries, float* grad2d, const gsr_backward_opts* opts,
                                          const uint8_t* block_mask, const uint32_t* tile_order,
                                          gsr_stream_t stream_) {
    gsr_backward_opts o = {GSR_REDUCE_WARP, 0, 1, 1, 2, {0, 0, 0}};
    if (opts) o = *opts;
    if (width <= 0 || height <= 0 || n < 0 || !tile_ranges || !splat2d || !bg || !dL_dimage || !grad2d)
        return GSR_EINVAL;
    if (n > 0 && (!radius || !entry_offsets || !partial || !point_list)) return GSR_EINVAL;
    if (partial_entries < 0) return GSR_EINVAL;
    if (!aligned16(splat2d) || !aligned16(grad2d) || !aligned8(tile_ranges)) return GSR_EINVAL;
    if (tile_w != 16 || tile_h != 16) return GSR_EINVAL;
    if ((o.lane_layout != 0 && o.lane_layout != 1) || (o.store_T != 0 && o.store_T != 1)) return GSR_EINVAL;
    if (o.pixels_per_thread < 0 || o.pixels_per_thread > 2) return GSR_EINVAL;
    if (o.store_T && (!final_T || !n_contrib)) return GSR_EINVAL;
    if (n == 0) return GSR_OK;
    BwdArgs a = {};
    a.g = RasterGeom{width, height, (width + 15) / 16, (height + 15) / 16};
    a.ranges = reinterpret_cast<const uint2*>(tile_ranges);
    a.point_list = point_list;
    a.splat2d = splat2d;
    a.bg0 = bg[0]; a.bg1 = bg[1]; a.bg2 = bg[2];
    a.final_T = final_T;
    a.n_contrib = n_contrib;
    a.dL_dimage = dL_dimage;
    a.grad2d = grad2d;
    a.radius = radius;
    a.entry_off = entry_offsets;
    a.partial = partial;
    a.order = tile_order;
    a.block_mask = block_mask;
    a.n = n;
    a.partial_cap = partial_entries > 0xffffffffll ? 0xffffffffu : (uint32_t)partial_entries;
    const int tiles = a.g.gx * a.g.gy;
    cudaStream_t s = (cudaStream_t)stream_;
    const bool st = o.store_T != 0;
    zero_partial_kernel<<<152 * 8, 256, 0, s>>>(n, entry_offsets, a.partial_cap, partial);
    int rc;
    if (o.pixels_per_thread == 2)
        rc = o.lane_layout ? launch_det_store<1, 2>(st, tiles, a, s) : launch_det_store<0, 2>(st, tiles, a, s);
    else
        rc = o.lane_layout ? launch_det_store<1, 1>(st, tiles, a, s) : launch_det_store<0, 1>(st, tiles, a, s);
    if (rc != GSR_OK) return rc;
    entries_reduce_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, entry_offsets, partial, a.partial_cap, grad2d);
    return check_launch();
}
