// Internal device/host helpers of libgsr (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsr.h"

namespace gsr {

constexpr float kDilation = 0.3f;       // screen-space covariance dilation
constexpr float kAlphaMax = 0.99f;      // alpha cap
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 0.0001f;        // transmittance stop
constexpr float kFrustum = 1.3f;        // clamp of x/z in the EWA Jacobian
constexpr float kLambdaFloor = 0.1f;    // floor of the eigenvalue discriminant
constexpr unsigned kFull = 0xffffffffu;

// Records the CUDA error text for gsr_last_cuda_error().
int cuda_fail(cudaError_t e);
// Checks the last launch; returns GSR_OK or GSR_ECUDA.
int check_launch();

inline bool pow2_in(int x, int lo, int hi) { return x >= lo && x <= hi && (x & (x - 1)) == 0; }
inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
inline bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

// Tile rectangle of a splat: the 3DGS bounding-box rule written with
// floor(u) so it is exact integer arithmetic ([x0,x1) x [y0,y1)).
__device__ __forceinline__ void tile_rect(float u, float v, int r, int gx, int gy, int tw_log2,
                                          int th_log2, int& x0, int& x1, int& y0, int& y1) {
    int fu = (int)floorf(u), fv = (int)floorf(v);
    int tw = 1 << tw_log2, th = 1 << th_log2;
    x0 = min(max((fu - r) >> tw_log2, 0), gx);
    x1 = min(max((fu + r + tw - 1) >> tw_log2, 0), gx);
    y0 = min(max((fv - r) >> th_log2, 0), gy);
    y1 = min(max((fv + r + th - 1) >> th_log2, 0), gy);
}

// Evaluation of one splat at one pixel with a fixed sequence of IEEE
// operations, so that the forward and the backward kernels take bit-identical
// skip decisions:  sigma = (A dx^2 + C dy^2)/2 + B dx dy, G = exp(-sigma),
// alpha = min(0.99, o G).  A pair is skipped when sigma < 0 or
// alpha < 1/255.
struct SplatEval {
    float dx, dy, dxx, dyy, dxy, sigma, G, alpha;
    bool capped;
};

__device__ __forceinline__ void splat_sigma(float u, float v, float A, float B, float C, float px, float py,
                                            SplatEval& e) {
    e.dx = __fsub_rn(u, px);
    e.dy = __fsub_rn(v, py);
    e.dxx = __fmul_rn(e.dx, e.dx);
    e.dyy = __fmul_rn(e.dy, e.dy);
    e.dxy = __fmul_rn(e.dx, e.dy);
    const float q = __fmaf_rn(C, e.dyy, __fmul_rn(A, e.dxx));
    e.sigma = __fmaf_rn(0.5f, q, __fmul_rn(B, e.dxy));
}

__device__ __forceinline__ void splat_alpha(float o, SplatEval& e) {
    e.G = __expf(-e.sigma);
    const float oG = __fmul_rn(o, e.G);
    e.capped = oG > kAlphaMax;
    e.alpha = e.capped ? kAlphaMax : oG;
}

// Returns false when the pair is skipped (G and alpha are then unset when
// sigma < 0).
__device__ __forceinline__ bool eval_splat(float u, float v, float A, float B, float C, float o,
                                           float px, float py, SplatEval& e) {
    splat_sigma(u, v, A, B, C, px, py, e);
    if (e.sigma < 0.0f) return false;
    splat_alpha(o, e);
    return e.alpha >= kAlphaMin;
}

// eval_splat without the early return: every field is set, and the result
// is eval_splat's.
__device__ __forceinline__ bool eval_splat_all(float u, float v, float A, float B, float C, float o, float px,
                                               float py, SplatEval& e) {
    splat_sigma(u, v, A, B, C, px, py, e);
    splat_alpha(o, e);
    return e.sigma >= 0.0f && e.alpha >= kAlphaMin;
}

// ---- two pixels of one column as float2 pairs -----------------------------
// Blackwell's packed FP32 instructions (FFMA2 / FMUL2 / FADD2) evaluate both
// components in one instruction, each rounded exactly as the scalar
// operation: the pair functions below give, per component, the bits of the
// scalar splat evaluation above.
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

struct SplatEval2 {
    float dx, dxx;                   // shared by the two pixels (same column)
    float2 dy, dyy, dxy, sigma, G, alpha;
    bool capped0, capped1;
};

// Pixels (px, py0) and (px, py1), given as px and npy = (-py0, -py1).
__device__ __forceinline__ void splat_sigma2(float u, float v, float A, float B, float C, float px, float2 npy,
                                             SplatEval2& e) {
    e.dx = __fsub_rn(u, px);
    e.dxx = __fmul_rn(e.dx, e.dx);
    e.dy = __fadd2_rn(bc2(v), npy);  // v - py: the negation is exact
    e.dyy = __fmul2_rn(e.dy, e.dy);
    e.dxy = __fmul2_rn(bc2(e.dx), e.dy);
    const float2 q = __ffma2_rn(bc2(C), e.dyy, bc2(__fmul_rn(A, e.dxx)));
    e.sigma = __ffma2_rn(bc2(0.5f), q, __fmul2_rn(bc2(B), e.dxy));
}

__device__ __forceinline__ void splat_alpha2(float o, SplatEval2& e) {
    e.G = make_float2(__expf(-e.sigma.x), __expf(-e.sigma.y));
    const float2 oG = __fmul2_rn(bc2(o), e.G);
    e.capped0 = oG.x > kAlphaMax;
    e.capped1 = oG.y > kAlphaMax;
    e.alpha = make_float2(e.capped0 ? kAlphaMax : oG.x, e.capped1 ? kAlphaMax : oG.y);
}

// eval_splat_all for both pixels: whether each pair passes.
__device__ __forceinline__ void eval_splat2_all(float u, float v, float A, float B, float C, float o, float px,
                                                float2 npy, SplatEval2& e, bool& hit0, bool& hit1) {
    splat_sigma2(u, v, A, B, C, px, npy, e);
    splat_alpha2(o, e);
    hit0 = e.sigma.x >= 0.0f && e.alpha.x >= kAlphaMin;
    hit1 = e.sigma.y >= 0.0f && e.alpha.y >= kAlphaMin;
}

// Sums 9 per-lane values over the full warp in 12 shuffles (instead of the
// 45 of nine butterflies): every halving step exchanges half of the values
// still held, so lanes end up owning different parameters.  On return, lane
// L holds the warp total of parameter reduce9_param(L) when that is <= 8.
// The adds of one level are independent and go in pairs through the packed
// FP32 unit (each component rounds as a scalar add would).
__device__ __forceinline__ float reduce9(const float v[9], int lane) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
    // a lane keeps one value of each pair and sends the other to its partner
    auto send = [](float x, float y, bool b) { return b ? x : y; };
    auto keep = [](float x, float y, bool b) { return b ? y : x; };
    auto xch = [](float x, int off) { return __shfl_xor_sync(kFull, x, off); };
    const float2 w01 = __fadd2_rn(make_float2(keep(v[0], v[1], b4), keep(v[2], v[3], b4)),
                                  make_float2(xch(send(v[0], v[1], b4), 16), xch(send(v[2], v[3], b4), 16)));
    const float2 w23 = __fadd2_rn(make_float2(keep(v[4], v[5], b4), keep(v[6], v[7], b4)),
                                  make_float2(xch(send(v[4], v[5], b4), 16), xch(send(v[6], v[7], b4), 16)));
    const float w4 = keep(v[8], 0.0f, b4) + xch(send(v[8], 0.0f, b4), 16);
    const float2 x01 = __fadd2_rn(make_float2(keep(w01.x, w01.y, b3), keep(w23.x, w23.y, b3)),
                                  make_float2(xch(send(w01.x, w01.y, b3), 8), xch(send(w23.x, w23.y, b3), 8)));
    const float x2 = keep(w4, 0.0f, b3) + xch(send(w4, 0.0f, b3), 8);
    const float2 y01 = __fadd2_rn(make_float2(keep(x01.x, x01.y, b2), keep(x2, 0.0f, b2)),
                                  make_float2(xch(send(x01.x, x01.y, b2), 4), xch(send(x2, 0.0f, b2), 4)));
    const float z = keep(y01.x, y01.y, b1) + xch(send(y01.x, y01.y, b1), 2);
    return z + xch(z, 1);
}

// Parameter index owned by lane L after reduce9 (>= 9: padding / duplicate).
__device__ __forceinline__ int reduce9_param(int lane) {
    int b1 = (lane >> 1) & 1, b2 = (lane >> 2) & 1, b3 = (lane >> 3) & 1, b4 = (lane >> 4) & 1;
    if (lane & 1) return 16;  // odd lanes hold a copy of the even lane's sum
    if (b1) return (b2 | b3 | b4) ? 16 : 8;
    return 4 * b2 + 2 * b3 + b4;
}

__device__ __forceinline__ void red_add(float* addr, float v) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(addr), "f"(v) : "memory");
}

// One vector red of four floats (addr 16-byte aligned).
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// Longest-first tile order (one CTA of kOrderThreads): a counting sort of
// the tile ids by decreasing bucket of their list length, the bucket being
// floor(log2 len) with the next two bits below the leading one (0 for empty
// lists).  cnt: kOrderBuckets words of shared memory.  The CTA's global
// writes to ranges before the call must be followed by __syncthreads().
constexpr int kOrderThreads = 1024;
constexpr int kOrderBuckets = 128;

__device__ __forceinline__ int order_bucket(uint32_t len) {
    if (len == 0) return 0;
    const int l2 = 31 - __clz(len);
    return l2 < 2 ? 1 + l2 : 4 * l2 + (int)((len >> (l2 - 2)) & 3u);
}

__device__ __forceinline__ void tile_order_block(int tiles, const uint2* ranges, uint32_t* __restrict__ order,
                                                 uint32_t* cnt) {
    for (int b = threadIdx.x; b < kOrderBuckets; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        atomicAdd(&cnt[kOrderBuckets - 1 - order_bucket(r.y - r.x)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the bucket counts, in place
        constexpr int PER = kOrderBuckets / 32;
        uint32_t v[PER], s = 0;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            v[j] = cnt[threadIdx.x * PER + j];
            s += v[j];
        }
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(kFull, incl, o);
            if ((int)threadIdx.x >= o) incl += x;
        }
        uint32_t run = incl - s;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            cnt[threadIdx.x * PER + j] = run;
            run += v[j];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
        const uint2 r = ranges[t];
        order[atomicAdd(&cnt[kOrderBuckets - 1 - order_bucket(r.y - r.x)], 1u)] = (uint32_t)t;
    }
}

// Bitonic sort of the warp's (key, src) pairs in ascending (key, src) order;
// lane L ends with the L-th pair.
__device__ __forceinline__ void warp_sort_pairs(uint32_t& key, uint32_t& src, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint32_t ok = __shfl_xor_sync(kFull, key, j);
            const uint32_t os = __shfl_xor_sync(kFull, src, j);
            const bool take_min = (((lane & k) == 0) == ((lane & j) == 0));
            const bool other_smaller = (ok < key) || (ok == key && os < src);
            if (take_min == other_smaller) {
                key = ok;
                src = os;
            }
        }
    }
}

}  // namespace gsr
