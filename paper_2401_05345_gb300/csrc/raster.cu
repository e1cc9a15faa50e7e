// Forward blend and backward blend + per-splat gradient accumulation.
//
// One CTA per screen tile, one thread per pixel.  The tile's depth-sorted
// splat list is staged through shared memory in batches of one entry per
// thread (coalesced id load, three 16-byte record loads per entry); every
// thread then walks the whole batch, so all 32 lanes of a warp evaluate the
// same splat at the same time -- the property that makes the warp-level
// reduction of the backward legal without a match (Sec. V-A2 requires all
// lanes to update the same primitive; here it holds by construction).
#include <cub/device/device_radix_sort.cuh>

#include "gsr_internal.cuh"

namespace gsr {
namespace {

struct RasterGeom {
    int W, H, gx, gy;
};

// Pixel of thread `tid` inside a TW x TH tile.
//   LAYOUT 0: row-major, a warp covers 32 consecutive pixels (16 x 2);
//   LAYOUT 1: each warp covers an 8 x 4 pixel block.
template <int TW, int LAYOUT>
__device__ __forceinline__ void lane_pixel(int tid, int& lx, int& ly) {
    if (LAYOUT == 0) {
        lx = tid % TW;
        ly = tid / TW;
    } else {
        const int w = tid >> 5, l = tid & 31;
        constexpr int WX = TW / 8;
        lx = (w % WX) * 8 + (l & 7);
        ly = (w / WX) * 4 + (l >> 3);
    }
}

// Bitmask of the warps of a TW x TH tile with origin (ox, oy) whose pixel
// block can hold a pixel where this splat reaches alpha >= 1/255.  Uses the
// bounding box of the ellipse sigma <= ln(255 o) (half-widths
// sqrt(2 L C / det), sqrt(2 L A / det) for the conic [[A,B],[B,C]]), with L
// enlarged by 1% + 0.01 and the box by 2% + 0.05 px, so FP32 rounding of
// sigma or alpha can never let a culled pair pass the alpha test: culling
// removes only pairs both kernels skip anyway.
template <int TW, int TH, int LAYOUT>
__device__ __forceinline__ unsigned warp_cull_mask(float u, float v, float A, float B, float C, float o,
                                                   int ox, int oy) {
    constexpr int NW = TW * TH / 32;
    constexpr unsigned ALL = NW >= 32 ? 0xffffffffu : ((1u << NW) - 1u);
    if (!(o >= kAlphaMin)) return 0u;  // alpha = o G <= o < 1/255 at every pixel
    const float det = A * C - B * B;
    if (!(det > 0.0f) || !(A > 0.0f) || !(C > 0.0f)) return ALL;
    const float L = __logf(o * 255.0f) * 1.01f + 0.01f;
    const float ex = sqrtf(2.0f * L * C / det) * 1.02f + 0.05f;
    const float ey = sqrtf(2.0f * L * A / det) * 1.02f + 0.05f;
    unsigned m = 0u;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        int x0, y0, wx, wy;
        if (LAYOUT == 0) {
            constexpr int RPW = 32 / TW;
            x0 = ox; y0 = oy + w * RPW; wx = TW; wy = RPW;
        } else {
            constexpr int WX = TW / 8;
            x0 = ox + (w % WX) * 8; y0 = oy + (w / WX) * 4; wx = 8; wy = 4;
        }
        const bool hit = (u + ex >= (float)x0) && (u - ex <= (float)(x0 + wx - 1)) &&
                         (v + ey >= (float)y0) && (v - ey <= (float)(y0 + wy - 1));
        m |= hit ? (1u << w) : 0u;
    }
    return m;
}

// Front-to-back walk of one pixel over its tile list (shared by the forward
// kernel and the recompute mode of the backward, so both produce the same
// final transmittance and last contributor bit for bit).  All threads of the
// CTA must call it.
template <int TW, int TH, int LAYOUT, bool COLOR>
__device__ __forceinline__ void walk_front(uint2 rg, const uint32_t* __restrict__ point_list,
                                           const float* __restrict__ splat2d, float px, float py,
                                           bool inside, int ox, int oy, float4* s_a, float4* s_b,
                                           float* s_c, unsigned* s_mask, float& T, int& last, float& C0,
                                           float& C1, float& C2) {
    constexpr int B = TW * TH;
    const int n = (int)(rg.y - rg.x);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    bool done = !inside;
    T = 1.0f;
    last = 0;
    C0 = C1 = C2 = 0.0f;
    for (int base = 0; base < n; base += B) {
        if (__syncthreads_count(done) == B) break;
        int idx = base + (int)threadIdx.x;
        if (idx < n) {
            uint32_t id = point_list[rg.x + idx];
            const float4* rec = reinterpret_cast<const float4*>(splat2d + (size_t)id * GSR_REC);
            const float4 a = rec[0], b = rec[1];
            s_a[threadIdx.x] = a;
            s_b[threadIdx.x] = b;
            if (COLOR) s_c[threadIdx.x] = rec[2].x;
            s_mask[threadIdx.x] = warp_cull_mask<TW, TH, LAYOUT>(a.x, a.y, a.z, a.w, b.x, b.y, ox, oy);
        }
        __syncthreads();
        const int cnt = min(B, n - base);
        bool wdone = __all_sync(kFull, done);
        for (int c0 = 0; c0 < cnt && !wdone; c0 += 32) {
            const int kq = c0 + lane;
            unsigned bits = __ballot_sync(kFull, kq < cnt && ((s_mask[kq] >> w) & 1u));
            while (bits) {
                const int k = c0 + __ffs(bits) - 1;
                bits &= bits - 1u;
                if (!done) {
                    const float4 a = s_a[k], b = s_b[k];
                    SplatEval e;
                    if (eval_splat(a.x, a.y, a.z, a.w, b.x, b.y, px, py, e)) {
                        const float testT = __fmul_rn(T, __fsub_rn(1.0f, e.alpha));
                        if (testT < kTMin) {
                            done = true;
                        } else {
                            if (COLOR) {
                                const float wgt = __fmul_rn(e.alpha, T);
                                C0 = __fmaf_rn(b.z, wgt, C0);
                                C1 = __fmaf_rn(b.w, wgt, C1);
                                C2 = __fmaf_rn(s_c[k], wgt, C2);
                            }
                            T = testT;
                            last = base + k + 1;
                        }
                    }
                }
                if (__all_sync(kFull, done)) {
                    wdone = true;
                    break;
                }
            }
        }
    }
}

template <int TW, int TH>
__global__ void __launch_bounds__(TW* TH)
forward_kernel(RasterGeom g, const uint2* __restrict__ ranges, const uint32_t* __restrict__ point_list,
               const float* __restrict__ splat2d, float bg0, float bg1, float bg2,
               float* __restrict__ image, float* __restrict__ final_T, int* __restrict__ n_contrib) {
    constexpr int B = TW * TH;
    __shared__ float4 s_a[B];
    __shared__ float4 s_b[B];
    __shared__ float s_c[B];
    __shared__ unsigned s_mask[B];
    const int tile = blockIdx.x;
    const int tx = tile % g.gx, ty = tile / g.gx;
    int lx, ly;
    lane_pixel<TW, 1>((int)threadIdx.x, lx, ly);
    const int px = tx * TW + lx, py = ty * TH + ly;
    const bool inside = px < g.W && py < g.H;
    float T, C0, C1, C2;
    int last;
    walk_front<TW, TH, 1, true>(ranges[tile], point_list, splat2d, (float)px, (float)py, inside, tx * TW,
                                ty * TH, s_a, s_b, s_c, s_mask, T, last, C0, C1, C2);
    if (inside) {
        const size_t HW = (size_t)g.W * g.H, pix = (size_t)py * g.W + px;
        image[pix] = __fmaf_rn(T, bg0, C0);
        image[HW + pix] = __fmaf_rn(T, bg1, C1);
        image[2 * HW + pix] = __fmaf_rn(T, bg2, C2);
        if (final_T) final_T[pix] = T;
        if (n_contrib) n_contrib[pix] = last;
    }
}

struct BwdArgs {
    RasterGeom g;
    const uint2* ranges;
    const uint32_t* point_list;
    const float* splat2d;
    float bg0, bg1, bg2;
    const float* final_T;
    const int* n_contrib;
    const float* dL_dimage;
    float* grad2d;
    int threshold;
};

template <int B, int MODE>
struct BwdSmem {
    float4 a[B];
    float4 b[B];
    float c[B];
    uint32_t id[B];
    unsigned mask[B];
    float acc[MODE == GSR_REDUCE_BLOCK ? B * 9 : 1];
    int maxlast;
};

// Backward of one tile: the gradient-computation step (Sec. III-A) for the
// tile's pixels, accumulated by the tier MODE.  All threads of the CTA call
// it; shared storage is reused across calls.
template <int TW, int TH, int MODE, int LAYOUT, bool STORE_T>
__device__ __forceinline__ void backward_tile(const BwdArgs& p, const int tile, BwdSmem<TW * TH, MODE>& sm) {
    constexpr int B = TW * TH;
    float4* s_a = sm.a;
    float4* s_b = sm.b;
    float* s_c = sm.c;
    uint32_t* s_id = sm.id;
    unsigned* s_mask = sm.mask;
    float* s_acc = sm.acc;
    int& s_maxlast = sm.maxlast;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tile % p.g.gx, ty = tile / p.g.gx;
    int lx, ly;
    lane_pixel<TW, LAYOUT>(tid, lx, ly);
    const int px = tx * TW + lx, py = ty * TH + ly;
    const bool inside = px < p.g.W && py < p.g.H;
    const float fpx = (float)px, fpy = (float)py;
    const uint2 rg = p.ranges[tile];
    const size_t HW = (size_t)p.g.W * p.g.H, pix = (size_t)py * p.g.W + px;

    float Tf;
    int last;
    const int nlist = (int)(rg.y - rg.x);
    if (STORE_T) {
        Tf = inside ? p.final_T[pix] : 0.0f;
        last = inside ? min(max(p.n_contrib[pix], 0), nlist) : 0;  // never walk past the list
    } else {
        float c0, c1, c2;
        walk_front<TW, TH, LAYOUT, false>(rg, p.point_list, p.splat2d, fpx, fpy, inside, tx * TW, ty * TH,
                                          s_a, s_b, s_c, s_mask, Tf, last, c0, c1, c2);
        if (!inside) { Tf = 0.0f; last = 0; }
    }
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (inside) {
        g0 = p.dL_dimage[pix];
        g1 = p.dL_dimage[HW + pix];
        g2 = p.dL_dimage[2 * HW + pix];
    }
    if (tid == 0) s_maxlast = 0;
    if (MODE == GSR_REDUCE_BLOCK)
        for (int i = tid; i < B * 9; i += B) s_acc[i] = 0.0f;
    __syncthreads();
    const int wlast = __reduce_max_sync(kFull, last);
    if (lane == 0) atomicMax(&s_maxlast, wlast);
    __syncthreads();
    const int maxlast = s_maxlast;

    float T = Tf;
    float S = Tf * (p.bg0 * g0 + p.bg1 * g1 + p.bg2 * g2);
    const int rparam = reduce9_param(lane);
    float* __restrict__ grad = p.grad2d;

    for (int top = maxlast; top > 0; top -= B) {
        const int cnt = min(B, top);
        __syncthreads();
        if (tid < cnt) {
            uint32_t id = p.point_list[rg.x + (uint32_t)(top - 1 - tid)];
            const float4* rec = reinterpret_cast<const float4*>(p.splat2d + (size_t)id * GSR_REC);
            const float4 a = rec[0], b = rec[1];
            s_id[tid] = id;
            s_a[tid] = a;
            s_b[tid] = b;
            s_c[tid] = rec[2].x;
            s_mask[tid] = warp_cull_mask<TW, TH, LAYOUT>(a.x, a.y, a.z, a.w, b.x, b.y, tx * TW, ty * TH);
        }
        __syncthreads();
        // each warp visits, back to front, only the staged splats whose
        // alpha >= 1/255 region touches its pixel block and that lie before
        // the warp's last contributor
        for (int c0 = 0; c0 < cnt; c0 += 32) {
          const int kq = c0 + lane;
          unsigned bits = __ballot_sync(kFull, kq < cnt && ((s_mask[kq] >> warp) & 1u) && (top - 1 - kq < wlast));
          while (bits) {
            const int k = c0 + __ffs(bits) - 1;
            bits &= bits - 1u;
            const int pos = top - 1 - k;
            const float4 a = s_a[k], b = s_b[k];
            SplatEval e;
            const bool active = (pos < last) && eval_splat(a.x, a.y, a.z, a.w, b.x, b.y, fpx, fpy, e);
            float v[9];
            if (active) {
                const float inv = __frcp_rn(1.0f - e.alpha);
                const float Tj = T * inv;
                const float cb = s_c[k];
                const float cg = b.z * g0 + b.w * g1 + cb * g2;
                const float dal = Tj * cg - S * inv;
                const float w = e.alpha * Tj;
                S = fmaf(cg, w, S);
                T = Tj;
                v[6] = w * g0;
                v[7] = w * g1;
                v[8] = w * g2;
                const float dsig = e.capped ? 0.0f : -b.y * e.G * dal;
                v[5] = e.capped ? 0.0f : e.G * dal;
                v[0] = (a.z * e.dx + a.w * e.dy) * dsig;
                v[1] = (a.w * e.dx + b.x * e.dy) * dsig;
                v[2] = 0.5f * e.dx * e.dx * dsig;
                v[3] = e.dx * e.dy * dsig;
                v[4] = 0.5f * e.dy * e.dy * dsig;
            } else {
#pragma unroll
                for (int q = 0; q < 9; ++q) v[q] = 0.0f;
            }
            float* rec = grad + (size_t)s_id[k] * GSR_REC;
            if (MODE == GSR_REDUCE_PLAIN) {
                if (active) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) atomicAdd(rec + q, v[q]);
                }
            } else {
                const unsigned m = __ballot_sync(kFull, active);
                if (m == 0u) continue;
                const bool dense = (MODE == GSR_REDUCE_WARP) || (__popc(m) >= p.threshold);
                if (dense) {
                    const float z = reduce9(v, lane);
                    if (rparam < 9) {
                        if (MODE == GSR_REDUCE_BLOCK) atomicAdd(&s_acc[k * 9 + rparam], z);
                        else red_add(rec + rparam, z);
                    }
                } else if (active) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        if (MODE == GSR_REDUCE_BLOCK) atomicAdd(&s_acc[k * 9 + q], v[q]);
                        else atomicAdd(rec + q, v[q]);
                    }
                }
            }
          }
        }
        if (MODE == GSR_REDUCE_BLOCK) {
            __syncthreads();
            for (int i = tid; i < cnt * 9; i += B) {
                const float val = s_acc[i];
                if (val != 0.0f) {
                    const int k = i / 9;
                    red_add(grad + (size_t)s_id[k] * GSR_REC + (i - 9 * k), val);
                    s_acc[i] = 0.0f;
                }
            }
        }
    }
}


template <int TW, int TH, int MODE, int LAYOUT, bool STORE_T>
__global__ void __launch_bounds__(TW* TH)
backward_kernel(BwdArgs p) {
    __shared__ BwdSmem<TW * TH, MODE> sm;
    backward_tile<TW, TH, MODE, LAYOUT, STORE_T>(p, blockIdx.x, sm);
}

// Persistent backward over many views: each CTA takes (view, tile) items in
// the given order (longest tile lists first) from one atomic counter until
// the list is exhausted.  No CTA waits on another.
template <int TW, int TH, int MODE, int LAYOUT, bool STORE_T>
__global__ void __launch_bounds__(TW* TH)
backward_batched_kernel(const gsr_view* __restrict__ views, const uint32_t* __restrict__ items, int n_items,
                        unsigned* __restrict__ counter, int threshold) {
    __shared__ BwdSmem<TW * TH, MODE> sm;
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const uint32_t code = items[it];
        const gsr_view& v = views[code >> 24];
        BwdArgs p;
        p.g = RasterGeom{v.width, v.height, (v.width + TW - 1) / TW, (v.height + TH - 1) / TH};
        p.ranges = reinterpret_cast<const uint2*>(v.tile_ranges);
        p.point_list = v.point_list;
        p.splat2d = v.splat2d;
        p.bg0 = v.bg[0]; p.bg1 = v.bg[1]; p.bg2 = v.bg[2];
        p.final_T = v.final_T;
        p.n_contrib = v.n_contrib;
        p.dL_dimage = v.dL_dimage;
        p.grad2d = v.grad2d;
        p.threshold = threshold;
        backward_tile<TW, TH, MODE, LAYOUT, STORE_T>(p, (int)(code & 0xffffffu), sm);
    }
}

// Counts of the backward traversal (no gradients written): per (warp, splat)
// step the number of active lanes -> hist[0..32]; hist[33] = active pairs,
// hist[34] = examined pairs (sum of n_contrib), hist[35] = warp steps with at
// least one lane still walking, hist[36] = those steps that pass the per-warp
// footprint cull, hist[37] = culled-in steps without any active lane.  The
// histogram is the active-lanes-per-warp measurement of Sec. III-B
// (Observation 2).
template <int TW, int TH, int LAYOUT>
__global__ void __launch_bounds__(TW* TH)
stats_kernel(BwdArgs p, unsigned long long* __restrict__ hist) {
    constexpr int B = TW * TH;
    __shared__ float4 s_a[B];
    __shared__ float4 s_b[B];
    __shared__ unsigned long long s_h[38];
    __shared__ unsigned s_mask[B];
    __shared__ int s_maxlast;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    const int tx = tile % p.g.gx, ty = tile / p.g.gx;
    int lx, ly;
    lane_pixel<TW, LAYOUT>(tid, lx, ly);
    const int px = tx * TW + lx, py = ty * TH + ly;
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
        if (tid < cnt) {
            uint32_t id = p.point_list[rg.x + (uint32_t)(top - 1 - tid)];
            const float4* rec = reinterpret_cast<const float4*>(p.splat2d + (size_t)id * GSR_REC);
            const float4 a = rec[0], b = rec[1];
            s_a[tid] = a;
            s_b[tid] = b;
            s_mask[tid] = warp_cull_mask<TW, TH, LAYOUT>(a.x, a.y, a.z, a.w, b.x, b.y, tx * TW, ty * TH);
        }
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

// Sort keys of the batched work order: larger tile lists first.
__global__ void batch_keys_kernel(int n_views, const gsr_view* __restrict__ views,
                                  const int* __restrict__ offsets, int n_items, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals) {
    __shared__ int s_off[257];
    for (int i = threadIdx.x; i <= n_views; i += blockDim.x) s_off[i] = offsets[i];
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_items; i += gridDim.x * blockDim.x) {
        int lo = 0, hi = n_views - 1;  // last view with offset <= i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const int t = i - s_off[lo];
        const uint32_t* r = views[lo].tile_ranges;
        const uint32_t len = r[2 * t + 1] - r[2 * t];
        keys[i] = 0xffffffffu - len;
        vals[i] = ((uint32_t)lo << 24) | (uint32_t)t;
    }
}

template <int MODE, int LAYOUT, bool STORE_T>
int launch_batched(int n_items, const gsr_view* views, const uint32_t* items, unsigned* counter, int thr,
                   int ctas_per_sm, cudaStream_t s) {
    auto k = backward_batched_kernel<16, 16, MODE, LAYOUT, STORE_T>;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    const int per_sm = ctas_per_sm > 0 ? min(ctas_per_sm, max(occ, 1)) : max(occ, 1);
    k<<<sms * per_sm, 256, 0, s>>>(views, items, n_items, counter, thr);
    return check_launch();
}

template <int MODE>
int launch_batched_mode(int layout, bool store, int n_items, const gsr_view* views, const uint32_t* items,
                        unsigned* counter, int thr, int cps, cudaStream_t s) {
    if (layout == 0)
        return store ? launch_batched<MODE, 0, true>(n_items, views, items, counter, thr, cps, s)
                     : launch_batched<MODE, 0, false>(n_items, views, items, counter, thr, cps, s);
    return store ? launch_batched<MODE, 1, true>(n_items, views, items, counter, thr, cps, s)
                 : launch_batched<MODE, 1, false>(n_items, views, items, counter, thr, cps, s);
}

template <int MODE, int LAYOUT, bool STORE_T>
void launch_bwd(int tiles, const BwdArgs& a, cudaStream_t s) {
    backward_kernel<16, 16, MODE, LAYOUT, STORE_T><<<tiles, 256, 0, s>>>(a);
}

template <int MODE>
void launch_bwd_mode(int layout, bool store, int tiles, const BwdArgs& a, cudaStream_t s) {
    if (layout == 0) {
        if (store) launch_bwd<MODE, 0, true>(tiles, a, s);
        else launch_bwd<MODE, 0, false>(tiles, a, s);
    } else {
        if (store) launch_bwd<MODE, 1, true>(tiles, a, s);
        else launch_bwd<MODE, 1, false>(tiles, a, s);
    }
}

}  // namespace
}  // namespace gsr

using namespace gsr;

extern "C" int gsr_forward(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                           const uint32_t* tile_ranges, const uint32_t* point_list, const float* splat2d,
                           const float* bg, float* image, float* final_T, int32_t* n_contrib,
                           gsr_stream_t stream) {
    if (width <= 0 || height <= 0 || !tile_ranges || !splat2d || !bg || !image) return GSR_EINVAL;
    if (!aligned16(splat2d) || !aligned8(tile_ranges)) return GSR_EINVAL;
    if (tile_w != 16 || tile_h != 16) return GSR_EINVAL;
    RasterGeom g{width, height, (width + 15) / 16, (height + 15) / 16};
    int tiles = g.gx * g.gy;
    forward_kernel<16, 16><<<tiles, 256, 0, (cudaStream_t)stream>>>(
        g, reinterpret_cast<const uint2*>(tile_ranges), point_list, splat2d, bg[0], bg[1], bg[2], image,
        final_T, n_contrib);
    return check_launch();
}

extern "C" int gsr_backward(int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                            const uint32_t* tile_ranges, const uint32_t* point_list, const float* splat2d,
                            const float* bg, const float* final_T, const int32_t* n_contrib,
                            const float* dL_dimage, float* grad2d, const gsr_backward_opts* opts,
                            gsr_stream_t stream_) {
    gsr_backward_opts o = {GSR_REDUCE_WARP, 0, 0, 1, {0, 0, 0, 0}};
    if (opts) o = *opts;
    if (width <= 0 || height <= 0 || !tile_ranges || !splat2d || !bg || !dL_dimage || !grad2d) return GSR_EINVAL;
    if (!aligned16(splat2d) || !aligned8(tile_ranges)) return GSR_EINVAL;
    if (tile_w != 16 || tile_h != 16) return GSR_EINVAL;
    if (o.reduce_mode < GSR_REDUCE_PLAIN || o.reduce_mode > GSR_REDUCE_BLOCK) return GSR_EINVAL;
    if (o.threshold < 0 || o.threshold > 33 || (o.lane_layout != 0 && o.lane_layout != 1)) return GSR_EINVAL;
    if (o.store_T != 0 && o.store_T != 1) return GSR_EINVAL;
    for (int i = 0; i < 4; ++i) if (o.reserved[i] != 0) return GSR_EINVAL;
    if (o.store_T && (!final_T || !n_contrib)) return GSR_EINVAL;
    BwdArgs a;
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
    const int tiles = a.g.gx * a.g.gy;
    cudaStream_t s = (cudaStream_t)stream_;
    const bool st = o.store_T != 0;
    switch (o.reduce_mode) {
        case GSR_REDUCE_PLAIN: launch_bwd_mode<GSR_REDUCE_PLAIN>(o.lane_layout, st, tiles, a, s); break;
        case GSR_REDUCE_WARP: launch_bwd_mode<GSR_REDUCE_WARP>(o.lane_layout, st, tiles, a, s); break;
        case GSR_REDUCE_HYBRID: launch_bwd_mode<GSR_REDUCE_HYBRID>(o.lane_layout, st, tiles, a, s); break;
        default: launch_bwd_mode<GSR_REDUCE_BLOCK>(o.lane_layout, st, tiles, a, s); break;
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
    if (lane_layout == 0) stats_kernel<16, 16, 0><<<tiles, 256, 0, s>>>(a, (unsigned long long*)hist);
    else stats_kernel<16, 16, 1><<<tiles, 256, 0, s>>>(a, (unsigned long long*)hist);
    return check_launch();
}

namespace gsr {
namespace {
size_t order_layout(int n_items, char* base, uint32_t** keys_in, uint32_t** keys_out, uint32_t** vals_in,
                    void** tmp, size_t* tmp_bytes) {
    size_t sort_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, (uint32_t*)nullptr, (uint32_t*)nullptr,
                                    (uint32_t*)nullptr, (uint32_t*)nullptr, n_items > 0 ? n_items : 1, 0, 32);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t vec = al(sizeof(uint32_t) * (size_t)(n_items > 0 ? n_items : 1));
    size_t off = 0;
    if (keys_in) *keys_in = base ? (uint32_t*)(base + off) : nullptr;
    off += vec;
    if (keys_out) *keys_out = base ? (uint32_t*)(base + off) : nullptr;
    off += vec;
    if (vals_in) *vals_in = base ? (uint32_t*)(base + off) : nullptr;
    off += vec;
    if (tmp) *tmp = base ? (void*)(base + off) : nullptr;
    if (tmp_bytes) *tmp_bytes = sort_bytes;
    return off + al(sort_bytes);
}
}  // namespace
}  // namespace gsr

extern "C" int gsr_batch_order_scratch_bytes(int32_t n_items, size_t* bytes) {
    if (n_items < 0 || !bytes) return GSR_EINVAL;
    *bytes = order_layout(n_items, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    return GSR_OK;
}

extern "C" int gsr_batch_order(int32_t n_views, const gsr_view* views, const int32_t* item_offsets,
                               int32_t n_items, void* scratch, size_t scratch_bytes, uint32_t* items_out,
                               gsr_stream_t stream_) {
    if (n_views <= 0 || n_views > 256 || n_items < 0 || !views || !item_offsets || !scratch || !items_out)
        return GSR_EINVAL;
    if (n_items == 0) return GSR_OK;
    uint32_t *kin, *kout, *vin;
    void* tmp;
    size_t tb;
    size_t need = order_layout(n_items, (char*)scratch, &kin, &kout, &vin, &tmp, &tb);
    if (scratch_bytes < need) return GSR_ESCRATCH;
    cudaStream_t s = (cudaStream_t)stream_;
    const int blocks = min((n_items + 255) / 256, 152 * 4);
    batch_keys_kernel<<<blocks, 256, 0, s>>>(n_views, views, item_offsets, n_items, kin, vin);
    int rc = check_launch();
    if (rc != GSR_OK) return rc;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(tmp, tb, kin, kout, vin, items_out, n_items, 0, 32, s);
    return e == cudaSuccess ? GSR_OK : cuda_fail(e);
}

extern "C" int gsr_backward_batched(int32_t n_views, const gsr_view* views, const uint32_t* items, int32_t n_items,
                                    uint32_t* counter, const gsr_backward_opts* opts, int32_t ctas_per_sm,
                                    gsr_stream_t stream_) {
    gsr_backward_opts o = {GSR_REDUCE_WARP, 0, 0, 1, {0, 0, 0, 0}};
    if (opts) o = *opts;
    if (n_views <= 0 || n_views > 256 || n_items < 0 || !views || !counter || (n_items > 0 && !items)) return GSR_EINVAL;
    if (o.reduce_mode < GSR_REDUCE_PLAIN || o.reduce_mode > GSR_REDUCE_BLOCK) return GSR_EINVAL;
    if (o.threshold < 0 || o.threshold > 33 || (o.lane_layout != 0 && o.lane_layout != 1)) return GSR_EINVAL;
    if ((o.store_T != 0 && o.store_T != 1) || ctas_per_sm < 0) return GSR_EINVAL;
    for (int i = 0; i < 4; ++i) if (o.reserved[i] != 0) return GSR_EINVAL;
    cudaStream_t s = (cudaStream_t)stream_;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (n_items == 0) return GSR_OK;
    const bool st = o.store_T != 0;
    unsigned* c = (unsigned*)counter;
    switch (o.reduce_mode) {
        case GSR_REDUCE_PLAIN:
            return launch_batched_mode<GSR_REDUCE_PLAIN>(o.lane_layout, st, n_items, views, items, c, o.threshold, ctas_per_sm, s);
        case GSR_REDUCE_WARP:
            return launch_batched_mode<GSR_REDUCE_WARP>(o.lane_layout, st, n_items, views, items, c, o.threshold, ctas_per_sm, s);
        case GSR_REDUCE_HYBRID:
            return launch_batched_mode<GSR_REDUCE_HYBRID>(o.lane_layout, st, n_items, views, items, c, o.threshold, ctas_per_sm, s);
        default:
            return launch_batched_mode<GSR_REDUCE_BLOCK>(o.lane_layout, st, n_items, views, items, c, o.threshold, ctas_per_sm, s);
    }
}
