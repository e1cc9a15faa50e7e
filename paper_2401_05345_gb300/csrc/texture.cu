// Cube-map texture sampling and the accumulation of its texture gradient:
// the second workload of the gradient-accumulation study, NvDiffRec's
// learning of an environment map from images (Sec. VI, "Workloads").  Each
// pixel samples the cube map bilinearly in its reflection direction; the
// backward adds w_k * dL/dout into the gradient of each of its 4 texels.
// Neighbouring pixels share texels, but the lanes of a warp update different
// texels (Sec. V-A1: the divergent case the serialized reduction SW-S is for),
// so the tiers are: per-lane scalar atomics (the baseline), per-lane vector
// reds, the serialized warp reduction over lanes that hit the same texel,
// a sorted segmented warp reduction, and a per-CTA shared-memory table.
#include "gsr_internal.cuh"

namespace gsr {
namespace {

constexpr int kTexTile = 16;        // CTA = 16 x 16 pixels, warp = 8 x 4 pixel block
constexpr int kTexThreads = 256;
constexpr uint32_t kNoTexel = 0xffffffffu;
constexpr int kTexSlots = 1024;     // shared table of the BLOCK tier
constexpr int kTexProbe = 8;

struct CubeTaps {
    uint32_t texel[4];  // face*R*R + row*R + column
    float w[4];
};

// Texel coordinates in FP32 with one rounding per listed operation (the
// oracle evaluates the same sequence), OpenGL cube-map faces and (s, t).
__device__ __forceinline__ bool cube_taps(float dx, float dy, float dz, int R, CubeTaps& t) {
    const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
    float sc, tc, ma;
    int face;
    if (ax >= ay && ax >= az) {
        ma = ax;
        face = dx >= 0.0f ? 0 : 1;
        sc = dx >= 0.0f ? -dz : dz;
        tc = -dy;
    } else if (ay >= az) {
        ma = ay;
        face = dy >= 0.0f ? 2 : 3;
        sc = dx;
        tc = dy >= 0.0f ? dz : -dz;
    } else {
        ma = az;
        face = dz >= 0.0f ? 4 : 5;
        sc = dz >= 0.0f ? dx : -dx;
        tc = -dy;
    }
    if (!(ma > 0.0f)) return false;
    const float fR = (float)R;
    const float s = __fmul_rn(__fadd_rn(__fdiv_rn(sc, ma), 1.0f), 0.5f);
    const float tt = __fmul_rn(__fadd_rn(__fdiv_rn(tc, ma), 1.0f), 0.5f);
    const float u = __fsub_rn(__fmul_rn(s, fR), 0.5f);
    const float v = __fsub_rn(__fmul_rn(tt, fR), 0.5f);
    const float u0 = floorf(u), v0 = floorf(v);
    const float fu = __fsub_rn(u, u0), fv = __fsub_rn(v, v0);
    const int x0 = (int)u0, y0 = (int)v0;
    const int xa = min(max(x0, 0), R - 1), xb = min(max(x0 + 1, 0), R - 1);
    const int ya = min(max(y0, 0), R - 1), yb = min(max(y0 + 1, 0), R - 1);
    const uint32_t base = (uint32_t)face * (uint32_t)R * (uint32_t)R;
    t.texel[0] = base + (uint32_t)(ya * R + xa);
    t.texel[1] = base + (uint32_t)(ya * R + xb);
    t.texel[2] = base + (uint32_t)(yb * R + xa);
    t.texel[3] = base + (uint32_t)(yb * R + xb);
    const float gu = 1.0f - fu, gv = 1.0f - fv;
    t.w[0] = gu * gv;
    t.w[1] = fu * gv;
    t.w[2] = gu * fv;
    t.w[3] = fu * fv;
    return true;
}

__global__ void __launch_bounds__(256)
cube_forward_kernel(long long n, const float* __restrict__ dirs, int R, const float4* __restrict__ tex,
                    float* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    CubeTaps t;
    float o0 = 0.0f, o1 = 0.0f, o2 = 0.0f;
    if (cube_taps(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], R, t)) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 x = tex[t.texel[k]];
            o0 = fmaf(t.w[k], x.x, o0);
            o1 = fmaf(t.w[k], x.y, o1);
            o2 = fmaf(t.w[k], x.z, o2);
        }
    }
    out[3 * i] = o0;
    out[3 * i + 1] = o1;
    out[3 * i + 2] = o2;
}

// Backward: one thread per pixel of a 16 x 16 tile.
template <int METHOD>
__global__ void __launch_bounds__(kTexThreads)
cube_backward_kernel(int W, int H, const float* __restrict__ dirs, const float* __restrict__ dL, int R,
                     float* __restrict__ grad, int threshold) {
    __shared__ uint32_t s_key[METHOD == GSR_TEX_BLOCK ? kTexSlots : 1];
    __shared__ float4 s_val[METHOD == GSR_TEX_BLOCK ? kTexSlots : 1];
    __shared__ float4 s_stage[METHOD == GSR_TEX_SERIAL ? kTexThreads / 32 : 1][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gxt = (W + kTexTile - 1) / kTexTile;
    const int px = (blockIdx.x % gxt) * kTexTile + (w & 1) * 8 + (lane & 7);
    const int py = (blockIdx.x / gxt) * kTexTile + (w >> 1) * 4 + (lane >> 3);
    const bool inside = px < W && py < H;
    const size_t i = (size_t)py * W + px;
    CubeTaps t;
    bool valid = inside && cube_taps(dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], R, t);
    float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
    if (valid) {
        g0 = dL[3 * i];
        g1 = dL[3 * i + 1];
        g2 = dL[3 * i + 2];
    }
    if (METHOD == GSR_TEX_BLOCK) {
        for (int q = threadIdx.x; q < kTexSlots; q += kTexThreads) {
            s_key[q] = kNoTexel;
            s_val[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        __syncthreads();
    }
    const unsigned vmask = __ballot_sync(kFull, valid);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t key = valid ? t.texel[k] : kNoTexel;
        const float wk = valid ? t.w[k] : 0.0f;
        const float a = wk * g0, b = wk * g1, c = wk * g2;
        float* dst = grad + 4 * (size_t)(valid ? key : 0u);
        if (METHOD == GSR_TEX_PLAIN) {
            if (valid) {
                atomicAdd(dst, a);
                atomicAdd(dst + 1, b);
                atomicAdd(dst + 2, c);
            }
        } else if (METHOD == GSR_TEX_PLAIN_V4) {
            if (valid) red_add_v4(dst, a, b, c, 0.0f);
        } else if (METHOD == GSR_TEX_SERIAL) {
            // lanes with the same texel form a group (match mask); a group of
            // at least `threshold` lanes is reduced at the SM (Sec. V-A1):
            // its lanes stage their values in shared memory and the group's
            // lowest lane adds them in lane order and sends one v4 red;
            // smaller groups send one v4 red per lane
            const unsigned peers = __match_any_sync(kFull, key) & vmask;
            const bool reduced = valid && __popc(peers) >= threshold;
            const unsigned rl = __ballot_sync(kFull, reduced);
            if (valid && !reduced) red_add_v4(dst, a, b, c, 0.0f);
            if (reduced) {
                s_stage[w][lane] = make_float4(a, b, c, 0.0f);
                __syncwarp(rl);
                if (lane == __ffs(peers) - 1) {
                    float sa = 0.0f, sb = 0.0f, sc = 0.0f;
                    for (unsigned m = peers; m; m &= m - 1u) {
                        const float4 v = s_stage[w][__ffs(m) - 1];
                        sa += v.x;
                        sb += v.y;
                        sc += v.z;
                    }
                    red_add_v4(dst, sa, sb, sc, 0.0f);
                }
                __syncwarp(rl);  // read before the next tap restages
            }
        } else if (METHOD == GSR_TEX_SORTED) {
            uint32_t sk = key, src = (uint32_t)lane;
            warp_sort_pairs(sk, src, lane);
            float ya = __shfl_sync(kFull, a, (int)src);
            float yb = __shfl_sync(kFull, b, (int)src);
            float yc = __shfl_sync(kFull, c, (int)src);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t kp = __shfl_up_sync(kFull, sk, o);
                const float ta = __shfl_up_sync(kFull, ya, o);
                const float tb = __shfl_up_sync(kFull, yb, o);
                const float tcv = __shfl_up_sync(kFull, yc, o);
                if (lane >= o && kp == sk) {
                    ya += ta;
                    yb += tb;
                    yc += tcv;
                }
            }
            const uint32_t kn = __shfl_down_sync(kFull, sk, 1);
            if ((lane == 31 || kn != sk) && sk != kNoTexel) red_add_v4(grad + 4 * (size_t)sk, ya, yb, yc, 0.0f);
        } else {  // GSR_TEX_BLOCK
            if (valid) {
                uint32_t h = (key * 0x9E3779B1u) >> 22;  // 10 bits: kTexSlots slots
                bool done = false;
                for (int pr = 0; pr < kTexProbe && !done; ++pr) {
                    const uint32_t old = atomicCAS(&s_key[h], kNoTexel, key);
                    if (old == kNoTexel || old == key) {
                        atomicAdd(&s_val[h].x, a);
                        atomicAdd(&s_val[h].y, b);
                        atomicAdd(&s_val[h].z, c);
                        done = true;
                    }
                    h = (h + 1u) & (kTexSlots - 1);
                }
                if (!done) red_add_v4(dst, a, b, c, 0.0f);
            }
        }
    }
    if (METHOD == GSR_TEX_BLOCK) {
        __syncthreads();
        for (int q = threadIdx.x; q < kTexSlots; q += kTexThreads) {
            const uint32_t key = s_key[q];
            if (key != kNoTexel) {
                const float4 v = s_val[q];
                red_add_v4(grad + 4 * (size_t)key, v.x, v.y, v.z, 0.0f);
            }
        }
    }
}

}  // namespace
}  // namespace gsr

using namespace gsr;

extern "C" int gsr_cube_forward(int32_t width, int32_t height, const float* dirs, int32_t R, const float* tex,
                                float* out, gsr_stream_t stream) {
    if (width <= 0 || height <= 0 || R <= 0 || !dirs || !tex || !out) return GSR_EINVAL;
    if (6ll * R * R >= (1ll << 31) || !aligned16(tex)) return GSR_EINVAL;
    const long long n = (long long)width * height;
    cube_forward_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
        n, dirs, R, reinterpret_cast<const float4*>(tex), out);
    return check_launch();
}

extern "C" int gsr_cube_backward(int32_t width, int32_t height, const float* dirs, const float* dL_dout, int32_t R,
                                 float* grad_tex, int32_t method, int32_t threshold, gsr_stream_t stream_) {
    if (width <= 0 || height <= 0 || R <= 0 || !dirs || !dL_dout || !grad_tex) return GSR_EINVAL;
    if (6ll * R * R >= (1ll << 31) || !aligned16(grad_tex)) return GSR_EINVAL;
    if (method < GSR_TEX_PLAIN || method > GSR_TEX_BLOCK || threshold < 0 || threshold > 33) return GSR_EINVAL;
    const unsigned blocks = (unsigned)(((width + kTexTile - 1) / kTexTile) * ((height + kTexTile - 1) / kTexTile));
    cudaStream_t s = (cudaStream_t)stream_;
    switch (method) {
        case GSR_TEX_PLAIN:
            cube_backward_kernel<GSR_TEX_PLAIN><<<blocks, kTexThreads, 0, s>>>(width, height, dirs, dL_dout, R,
                                                                               grad_tex, threshold);
            break;
        case GSR_TEX_PLAIN_V4:
            cube_backward_kernel<GSR_TEX_PLAIN_V4><<<blocks, kTexThreads, 0, s>>>(width, height, dirs, dL_dout, R,
                                                                                  grad_tex, threshold);
            break;
        case GSR_TEX_SERIAL:
            cube_backward_kernel<GSR_TEX_SERIAL><<<blocks, kTexThreads, 0, s>>>(width, height, dirs, dL_dout, R,
                                                                                grad_tex, threshold);
            break;
        case GSR_TEX_SORTED:
            cube_backward_kernel<GSR_TEX_SORTED><<<blocks, kTexThreads, 0, s>>>(width, height, dirs, dL_dout, R,
                                                                                grad_tex, threshold);
            break;
        default:
            cube_backward_kernel<GSR_TEX_BLOCK><<<blocks, kTexThreads, 0, s>>>(width, height, dirs, dL_dout, R,
                                                                               grad_tex, threshold);
            break;
    }
    return check_launch();
}
