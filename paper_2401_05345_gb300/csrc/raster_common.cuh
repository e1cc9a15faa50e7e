// Shared device code of the forward and backward blend kernels.
//
// One CTA per 16x16 screen tile.  The tile's depth-sorted splat list is
// staged through shared memory in batches of one entry per pixel (coalesced
// id load, three 16-byte record loads per entry, and a per-warp cull mask);
// every warp then visits the staged splats that can touch its pixel block,
// all 32 lanes on the same splat at the same time -- the property that makes
// the warp-level reduction of the backward legal without a match (Sec. V-A2
// requires all lanes to update the same primitive; here it holds by
// construction).  Each thread owns PPT pixels of the tile.
#pragma once

#include "gsr_internal.cuh"

namespace gsr {

struct RasterGeom {
    int W, H, gx, gy;
};

// Thread / warp / pixel geometry of a TW x TH tile with PPT pixels per thread.
//   LAYOUT 0: a warp covers TW x (32 PPT / TW) consecutive rows;
//   LAYOUT 1: a warp covers an 8 x (4 PPT) pixel block.
// Pixel q of a lane lies 32/TW (LAYOUT 0) or 4 (LAYOUT 1) rows below pixel 0.
template <int TW, int TH, int LAYOUT, int PPT>
struct Shape {
    static constexpr int TWd = TW, THd = TH;
    static constexpr int B = TW * TH;       // pixels per tile = entries staged per batch
    static constexpr int NT = B / PPT;      // threads per CTA
    static constexpr int NW = NT / 32;      // warps per CTA
    static constexpr int BX = LAYOUT == 0 ? TW : 8;
    static constexpr int BY = LAYOUT == 0 ? 32 * PPT / TW : 4 * PPT;
    static constexpr int WX = TW / BX;      // warp blocks per tile row
    static_assert(B % PPT == 0 && NT % 32 == 0, "tile shape");

    __device__ static void pixel(int tid, int q, int& lx, int& ly) {
        const int w = tid >> 5, l = tid & 31;
        if (LAYOUT == 0) {
            lx = l % TW;
            ly = w * BY + l / TW + q * (32 / TW);
        } else {
            lx = (w % WX) * 8 + (l & 7);
            ly = (w / WX) * BY + (l >> 3) + 4 * q;
        }
    }
    __device__ static void warp_origin(int w, int& x0, int& y0) {
        x0 = (w % WX) * BX;
        y0 = (w / WX) * BY;
    }
};

// Bitmask of the warps of a tile (origin ox, oy) whose pixel block can hold
// a pixel where this splat reaches alpha >= 1/255, i.e. sigma <= ln(255 o).
// Two tests, both conservative: the bounding box of that ellipse
// (half-widths sqrt(2 L C / det), sqrt(2 L A / det) for the conic
// [[A,B],[B,C]]; box enlarged by 2% + 0.05 px), then the exact minimum of
// sigma over the warp's block (enlarged by 0.05 px): sigma is a convex
// quadratic, so when the centre lies outside the block the minimum is on an
// edge whose side the centre is on, at the clamped stationary point of that
// edge.  L is enlarged by 1% + 0.01 and the minimum is compared with
// L + 1e-5 (A X^2 + C Y^2 + 2 |B| X Y) (X, Y the block's extents from the
// centre), far above the FP32 rounding of either evaluation of sigma, so a
// culled pair can never pass the alpha test: culling removes only pairs
// every kernel skips.  The reciprocals and square roots are the hardware
// approximations (a few ulp): far inside those margins, and an inexact
// stationary point moves sigma only at second order.
template <class SH>
__device__ __forceinline__ unsigned warp_cull_mask(float u, float v, float A, float B, float C, float o, int ox,
                                                   int oy) {
    constexpr int NW = SH::NW;
    constexpr unsigned ALL = NW >= 32 ? 0xffffffffu : ((1u << NW) - 1u);
    if (!(o >= kAlphaMin)) return 0u;  // alpha = o G <= o < 1/255 at every pixel
    const float det = A * C - B * B;
    if (!(det > 0.0f) || !(A > 0.0f) || !(C > 0.0f)) return ALL;
    const float L = __logf(o * 255.0f) * 1.01f + 0.01f;
    const float iA = __fdividef(1.0f, A), iC = __fdividef(1.0f, C);
    const float t = __fdividef(2.0f * L, det);  // > 0
    const float tx = t * C, ty = t * A;
    const float ex = tx * rsqrtf(tx) * 1.02f + 0.05f;
    const float ey = ty * rsqrtf(ty) * 1.02f + 0.05f;
    const float fox = (float)ox, foy = (float)oy;  // pixel coordinates: integers, exact in FP32
    unsigned m = 0u;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        int bx, by;
        SH::warp_origin(w, bx, by);
        const float x0 = fox + (float)bx, x1 = fox + (float)(bx + SH::BX - 1);
        const float y0 = foy + (float)by, y1 = foy + (float)(by + SH::BY - 1);
        bool hit = (u + ex >= x0) && (u - ex <= x1) && (v + ey >= y0) && (v - ey <= y1);
        if (hit) {
            const float dxa = x0 - 0.05f - u, dxb = x1 + 0.05f - u;
            const float dya = y0 - 0.05f - v, dyb = y1 + 0.05f - v;
            if (dxa > 0.0f || dxb < 0.0f || dya > 0.0f || dyb < 0.0f) {  // centre outside the block
                float smin = 3.0e38f;
                if (dxa > 0.0f || dxb < 0.0f) {
                    const float X = dxa > 0.0f ? dxa : dxb;
                    const float Y = fminf(fmaxf(-B * X * iC, dya), dyb);
                    smin = fminf(smin, 0.5f * (A * X * X + C * Y * Y) + B * X * Y);
                }
                if (dya > 0.0f || dyb < 0.0f) {
                    const float Y = dya > 0.0f ? dya : dyb;
                    const float X = fminf(fmaxf(-B * Y * iA, dxa), dxb);
                    smin = fminf(smin, 0.5f * (A * X * X + C * Y * Y) + B * X * Y);
                }
                const float xm = fmaxf(fabsf(dxa), fabsf(dxb)), ym = fmaxf(fabsf(dya), fabsf(dyb));
                const float tol = 1e-5f * (A * xm * xm + C * ym * ym + 2.0f * fabsf(B) * xm * ym);
                hit = smin <= L + tol;
            }
        }
        m |= hit ? (1u << w) : 0u;
    }
    return m;
}

// Whether a tile shape's warps own the 2 x 2 blocks of 8 x 8 pixels that the
// per-entry block masks of gsr_forward / gsr_backward describe (bit w: block
// w, row-major in the tile).
template <class SH>
struct HasBlockMask {
    static constexpr bool value = SH::NW == 4 && SH::BX == 8 && SH::BY == 8 && SH::WX == 2;
};

// Stages batch entries [0, cnt) (list positions given by pos_of) into shared
// memory; with PPT > 1 every thread stages several entries.  The per-warp
// cull mask of an entry is read from mask_in when given (shapes with 8 x 8
// warp blocks), else computed, and then also written to mask_out when given.
template <class SH, bool COLOR, bool IDS, class PosOf>
__device__ __forceinline__ void stage_batch(int cnt, PosOf pos_of, const uint32_t* __restrict__ point_list,
                                            const float* __restrict__ splat2d, int ox, int oy, float4* s_a,
                                            float4* s_b, float* s_c, uint32_t* s_id, unsigned* s_mask,
                                            const uint8_t* __restrict__ mask_in, uint8_t* __restrict__ mask_out) {
    constexpr bool BM = HasBlockMask<SH>::value;
    for (int e = threadIdx.x; e < cnt; e += SH::NT) {
        const uint32_t pe = pos_of(e);
        const uint32_t id = point_list[pe];
        const float4* rec = reinterpret_cast<const float4*>(splat2d + (size_t)id * GSR_REC);
        const float4 a = rec[0], b = rec[1];
        s_a[e] = a;
        s_b[e] = b;
        if (COLOR) s_c[e] = rec[2].x;
        if (IDS) s_id[e] = id;
        unsigned mk;
        if (BM && mask_in) {
            mk = mask_in[pe];
        } else {
            mk = warp_cull_mask<SH>(a.x, a.y, a.z, a.w, b.x, b.y, ox, oy);
            if (BM && mask_out) mask_out[pe] = (uint8_t)mk;
        }
        s_mask[e] = mk;
    }
}

// Front-to-back walk of each of the thread's pixels over the tile list (the
// forward rule; shared by the forward kernel and the recompute mode of the
// backward, so both produce the same final transmittance and last
// contributor bit for bit).  All threads of the CTA must call it.
template <class SH, bool COLOR>
__device__ __forceinline__ void walk_front(uint2 rg, const uint32_t* __restrict__ point_list,
                                           const float* __restrict__ splat2d, const float* px, const float* py,
                                           const bool* inside, int ox, int oy, float4* s_a, float4* s_b,
                                           float* s_c, unsigned* s_mask, float* T, int* last, float (*C)[3],
                                           const uint8_t* mask_in, uint8_t* mask_out) {
    constexpr int PPT = SH::B / SH::NT;
    const int n = (int)(rg.y - rg.x);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    bool done[PPT];
    bool all_done = true;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        done[q] = !inside[q];
        all_done &= done[q];
        T[q] = 1.0f;
        last[q] = 0;
        C[q][0] = C[q][1] = C[q][2] = 0.0f;
    }
    // two pixels per thread share their column (Shape::pixel): their
    // transmittance and colour run as float2 pairs
    float2 T2 = bc2(1.0f), C2[3] = {bc2(0.0f), bc2(0.0f), bc2(0.0f)};
    // a pixel that is done (outside the image, or stopped) has a NaN row:
    // every splat's sigma is then NaN there and fails sigma >= 0, so the
    // hit test needs no done flag
    const float row_done = __int_as_float(0x7fc00000);  // a quiet NaN
    float2 npy = make_float2(inside[0] ? -py[0] : row_done, inside[PPT - 1] ? -py[PPT - 1] : row_done);
    for (int base = 0; base < n; base += SH::B) {
        if (__syncthreads_count(all_done) == SH::NT) break;
        const int cnt = min(SH::B, n - base);
        stage_batch<SH, COLOR, false>(cnt, [&](int e) { return rg.x + (uint32_t)(base + e); }, point_list,
                                      splat2d, ox, oy, s_a, s_b, s_c, nullptr, s_mask, mask_in, mask_out);
        __syncthreads();
        bool wdone = __all_sync(kFull, all_done);
        for (int c0 = 0; c0 < cnt && !wdone; c0 += 32) {
            // ballot bit 31 - i is entry c0 + i: the next entry is the highest set
            // bit (one ALU instruction fewer per step than the lowest; the ALU
            // pipe is what limits this walk)
            const int kq = c0 + 31 - lane;
            unsigned bits = __ballot_sync(kFull, kq < cnt && ((s_mask[kq] >> w) & 1u));
            while (bits) {
                const int lz = __clz(bits);
                const int k = c0 + lz;
                bits ^= 0x80000000u >> lz;
                const float4 a = s_a[k], b = s_b[k];
                const float cz = COLOR ? s_c[k] : 0.0f;
                // no branches: a pixel that is done or skips the splat keeps
                // T, last and C (its blend weight is 0)
                if constexpr (PPT == 2) {
                    SplatEval2 e;
                    bool hit0, hit1;
                    splat_sigma2(a.x, a.y, a.z, a.w, b.x, px[0], npy, e);
                    // alpha as in splat_alpha2, with the cap as a min (no capped
                    // flags: only the backward needs them)
                    const float2 oG = __fmul2_rn(bc2(b.y), make_float2(__expf(-e.sigma.x), __expf(-e.sigma.y)));
                    const float2 alpha = make_float2(fminf(oG.x, kAlphaMax), fminf(oG.y, kAlphaMax));
                    hit0 = e.sigma.x >= 0.0f && alpha.x >= kAlphaMin;
                    hit1 = e.sigma.y >= 0.0f && alpha.y >= kAlphaMin;
                    const float2 testT = __fmul2_rn(T2, __fadd2_rn(bc2(1.0f), neg2(alpha)));
                    const bool stop0 = hit0 && testT.x < kTMin, stop1 = hit1 && testT.y < kTMin;
                    const bool take0 = hit0 && !stop0, take1 = hit1 && !stop1;
                    npy.x = stop0 ? row_done : npy.x;
                    npy.y = stop1 ? row_done : npy.y;
                    // a pixel that does not take the splat blends it with alpha 0:
                    // weight 0 and T * (1 - 0) = T exactly, so T needs no select
                    const float2 ae = make_float2(take0 ? alpha.x : 0.0f, take1 ? alpha.y : 0.0f);
                    if (COLOR) {
                        const float2 wgt = __fmul2_rn(ae, T2);
                        C2[0] = __ffma2_rn(bc2(b.z), wgt, C2[0]);
                        C2[1] = __ffma2_rn(bc2(b.w), wgt, C2[1]);
                        C2[2] = __ffma2_rn(bc2(cz), wgt, C2[2]);
                    }
                    T2 = __fmul2_rn(T2, __fadd2_rn(bc2(1.0f), neg2(ae)));
                    last[0] = take0 ? base + k + 1 : last[0];
                    last[1] = take1 ? base + k + 1 : last[1];
                } else {
#pragma unroll
                    for (int q = 0; q < PPT; ++q) {
                        SplatEval e;
                        const bool hit = eval_splat_all(a.x, a.y, a.z, a.w, b.x, b.y, px[q], py[q], e) && !done[q];
                        const float testT = __fmul_rn(T[q], __fsub_rn(1.0f, e.alpha));
                        const bool stop = hit && testT < kTMin;
                        const bool take = hit && !stop;
                        done[q] = done[q] || stop;
                        if (COLOR) {
                            const float wgt = take ? __fmul_rn(e.alpha, T[q]) : 0.0f;
                            C[q][0] = __fmaf_rn(b.z, wgt, C[q][0]);
                            C[q][1] = __fmaf_rn(b.w, wgt, C[q][1]);
                            C[q][2] = __fmaf_rn(cz, wgt, C[q][2]);
                        }
                        T[q] = take ? testT : T[q];
                        last[q] = take ? base + k + 1 : last[q];
                    }
                }
            }
            if constexpr (PPT == 2) {
                all_done = isnan(npy.x) && isnan(npy.y);
            } else {
                all_done = true;
#pragma unroll
                for (int q = 0; q < PPT; ++q) all_done &= done[q];
            }
            wdone = __all_sync(kFull, all_done);
        }
    }
    if constexpr (PPT == 2) {
        T[0] = T2.x;
        T[1] = T2.y;
        if (COLOR) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                C[0][ch] = C2[ch].x;
                C[1][ch] = C2[ch].y;
            }
        }
    }
}

struct BwdArgs {
    RasterGeom g;
    const uint32_t* order;  // tile of CTA b: order[b] (NULL: b)
    const uint2* ranges;
    const uint32_t* point_list;
    const float* splat2d;
    float bg0, bg1, bg2;
    const float* final_T;
    const int* n_contrib;
    const float* dL_dimage;
    float* grad2d;
    int threshold;
    // deterministic tier only
    const int* radius;
    const uint32_t* entry_off;
    float* partial;
    int n;                // Gaussians (entry_off has n + 1 values)
    uint32_t partial_cap; // entries partial holds
    const uint8_t* block_mask;  // per-entry cull masks from the forward, or NULL
    // count mode only
    unsigned long long* counts;  // kCountSlots totals, see kModeCount
    int count_tier;              // tier whose global reds are counted (PLAIN, WARP or HYBRID)
};

// Count mode: the traversal of a tier (count_tier, threshold) with every
// global red replaced by counting it.  counts[0] scalar red warp
// instructions, [1] vector (v4) red warp instructions, [2] floats added at
// L2, [3] lane-level red operations (what the L2 receives before any
// coalescing), [4] (warp, splat) steps walked, [5] of those with an active
// lane, [6 + a] steps with exactly a active lanes (a = 0..32).
constexpr int kModeCount = 6;
constexpr int kCountSlots = 6 + 33;

// Deterministic tier: per-warp partial sums are combined in warp order and
// written, without atomics, to one 9-float slot per (tile, splat) list entry
// that some pixel of the tile reaches (the other slots keep the zeros they
// were cleared to before the launch).
constexpr int kModeDet = 4;
// Staged entries whose per-warp sums are combined at a time: the per-warp
// sums of 64 entries (9 KB for 4 warps) instead of a whole 256-entry batch
// let more CTAs share an SM.
constexpr int kDetGroup = 64;

// Shared arrays of the deterministic tier (dynamic shared memory).
struct DetSmem {
    float* part;        // [warps][B][9] per-warp partial sums of the batch
    unsigned* wflags;   // [B] warps that wrote a partial for entry k
};

// Cluster tier: a 2 x 2 cluster of tile CTAs pre-reduces its warps' splat
// gradients in a hash table spread over the four CTAs' shared memory
// (distributed shared memory); every splat id has one owner CTA and one slot
// there, and each CTA flushes its part with one global red per (cluster,
// splat, parameter) once the whole cluster is done.
constexpr int kModeCluster = 5;
constexpr uint32_t kSlotEmpty = 0xffffffffu;
constexpr int kClusterProbe = 16;  // slots tried before falling back to a global red

struct ClusterTab {
    uint32_t key_base;  // shared::cta addresses of this CTA's key[cap] (every
    uint32_t val_base;  // CTA of the cluster has them at the same offsets) and val[cap][9]
    int cap;            // slots per CTA (a power of two)
};

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address, in the cluster's shared window, of shared::cta address `la` of
// CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_map(uint32_t la, uint32_t rank) {
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(rank));
    return ra;
}

__device__ __forceinline__ uint32_t dsm_cas(uint32_t addr, uint32_t cmp, uint32_t val) {
    uint32_t old;
    asm volatile("atom.shared::cluster.cas.b32 %0, [%1], %2, %3;" : "=r"(old) : "r"(addr), "r"(cmp), "r"(val)
                 : "memory");
    return old;
}

__device__ __forceinline__ void dsm_red_add(uint32_t addr, float v) {
    asm volatile("red.shared::cluster.add.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// Every thread of every CTA of the cluster: writes before it are visible to
// the cluster after it.
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Slot of splat `id` in the cluster table (claimed if new), as (owner CTA,
// slot), or -1 when kClusterProbe slots are taken by other ids.
__device__ __forceinline__ int cluster_slot(const ClusterTab& ct, uint32_t id, uint32_t& owner) {
    const uint32_t h = id * 0x9E3779B1u;
    owner = h >> 30;
    uint32_t s = (h >> 8) & (uint32_t)(ct.cap - 1);
    for (int pr = 0; pr < kClusterProbe; ++pr) {
        const uint32_t old = dsm_cas(cluster_map(ct.key_base + 4u * s, owner), kSlotEmpty, id);
        if (old == kSlotEmpty || old == id) return (int)s;
        s = (s + 1u) & (uint32_t)(ct.cap - 1);
    }
    return -1;
}

// Slot of the (tile, Gaussian) entry in the per-Gaussian layout: the
// Gaussian's first slot plus the tile's row-major rank inside its rectangle
// (the order binning emits the entries in).
__device__ __forceinline__ uint32_t entry_slot(const BwdArgs& p, uint32_t id, float u, float v, int tile) {
    int x0, x1, y0, y1;
    tile_rect(u, v, p.radius[id], p.g.gx, p.g.gy, 4, 4, x0, x1, y0, y1);
    const int tx = tile % p.g.gx, ty = tile / p.g.gx;
    return p.entry_off[id] + (uint32_t)((ty - y0) * (x1 - x0) + (tx - x0));
}

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

// Gradients of one active (pixel, splat) pair, walking back to front, added
// to v[0..9): T holds T_{j+1} on entry and T_j on exit; S accumulates
// sum_{k>j} (c_k . g) alpha_k T_k + T_final (bg . g).  With
// dL/dalpha = T_j (c_j . g) - S / (1 - alpha_j):  dL/dc = alpha T_j g,
// dL/do = G dL/dalpha, dL/dsigma = -o G dL/dalpha (both 0 where alpha is
// capped), and through sigma = (A dx^2 + C dy^2)/2 + B dx dy:
// dL/d(u, v) = (A dx + B dy, B dx + C dy) dL/dsigma,
// dL/d(A, B, C) = (dx^2/2, dx dy, dy^2/2) dL/dsigma.  Every output is one
// fused multiply-add into its running sum.
template <bool FIRST>
__device__ __forceinline__ void pair_grads(const SplatEval& e, float4 a, float4 b, float cb, float g0, float g1,
                                           float g2, float& T, float& S, float* v) {
    // 1 / (1 - alpha), 1 - alpha in [0.01, 1): the hardware reciprocal
    // estimate refined by one Newton-Raphson step r <- r + r (1 - d r), which
    // squares the estimate's relative error (a few ulp before the step)
    const float d = 1.0f - e.alpha;
    float inv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv) : "f"(d));
    inv = fmaf(inv, fmaf(-d, inv, 1.0f), inv);
    const float Tj = T * inv;
    const float cg = fmaf(b.z, g0, fmaf(b.w, g1, cb * g2));
    const float dal = fmaf(Tj, cg, -S * inv);
    const float w = e.alpha * Tj;
    S = fmaf(cg, w, S);
    T = Tj;
    const float dop = e.capped ? 0.0f : e.G * dal;
    const float dsig = -b.y * dop;
    const float hd = 0.5f * dsig;
    const float du = fmaf(a.z, e.dx, a.w * e.dy), dv = fmaf(a.w, e.dx, b.x * e.dy);
    if (FIRST) {  // the first pixel slot writes the lane's sums
        v[6] = w * g0;
        v[7] = w * g1;
        v[8] = w * g2;
        v[5] = dop;
        v[0] = du * dsig;
        v[1] = dv * dsig;
        v[2] = e.dxx * hd;
        v[3] = e.dxy * dsig;
        v[4] = e.dyy * hd;
    } else {
        v[6] = fmaf(w, g0, v[6]);
        v[7] = fmaf(w, g1, v[7]);
        v[8] = fmaf(w, g2, v[8]);
        v[5] += dop;
        v[0] = fmaf(du, dsig, v[0]);
        v[1] = fmaf(dv, dsig, v[1]);
        v[2] = fmaf(e.dxx, hd, v[2]);
        v[3] = fmaf(e.dxy, dsig, v[3]);
        v[4] = fmaf(e.dyy, hd, v[4]);
    }
}

// pair_grads for the two pixels of one column as float2 pairs (Blackwell's
// packed FFMA2 / FMUL2 / FADD2): per component the operations of pair_grads,
// so the bits of two scalar calls.  act0 / act1 select the active pairs
// (alpha and G enter as 0 otherwise); the 9 sums of the two pixels are
// written to v.
__device__ __forceinline__ void pair_grads2(const SplatEval2& e, bool act0, bool act1, float4 a, float4 b, float cb,
                                            float2 g0, float2 g1, float2 g2, float2& T, float2& S, float* v) {
    const float2 al = make_float2(act0 ? e.alpha.x : 0.0f, act1 ? e.alpha.y : 0.0f);
    // G for dL/do: 0 where the pair is inactive or alpha is capped
    const float2 Gd = make_float2(act0 && !e.capped0 ? e.G.x : 0.0f, act1 && !e.capped1 ? e.G.y : 0.0f);
    const float2 d = __fadd2_rn(bc2(1.0f), neg2(al));
    float2 inv;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv.x) : "f"(d.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(inv.y) : "f"(d.y));
    inv = __ffma2_rn(inv, __ffma2_rn(neg2(d), inv, bc2(1.0f)), inv);
    const float2 Tj = __fmul2_rn(T, inv);
    const float2 cg = __ffma2_rn(bc2(b.z), g0, __ffma2_rn(bc2(b.w), g1, __fmul2_rn(bc2(cb), g2)));
    const float2 dal = __ffma2_rn(Tj, cg, neg2(__fmul2_rn(S, inv)));
    const float2 w = __fmul2_rn(al, Tj);
    S = __ffma2_rn(cg, w, S);
    T = Tj;
    const float2 dop = __fmul2_rn(Gd, dal);
    const float2 dsig = __fmul2_rn(bc2(-b.y), dop);
    const float2 hd = __fmul2_rn(bc2(0.5f), dsig);
    const float2 du = __ffma2_rn(bc2(a.z), bc2(e.dx), __fmul2_rn(bc2(a.w), e.dy));
    const float2 dv = __ffma2_rn(bc2(a.w), bc2(e.dx), __fmul2_rn(bc2(b.x), e.dy));
    v[6] = fmaf(w.y, g0.y, w.x * g0.x);
    v[7] = fmaf(w.y, g1.y, w.x * g1.x);
    v[8] = fmaf(w.y, g2.y, w.x * g2.x);
    v[5] = dop.x + dop.y;
    v[0] = fmaf(du.y, dsig.y, du.x * dsig.x);
    v[1] = fmaf(dv.y, dsig.y, dv.x * dsig.x);
    v[2] = fmaf(e.dxx, hd.y, e.dxx * hd.x);
    v[3] = fmaf(e.dxy.y, dsig.y, e.dxy.x * dsig.x);
    v[4] = fmaf(e.dyy.y, hd.y, e.dyy.x * hd.x);
}

// Backward of one tile: the gradient-computation step (Sec. III-A) for the
// tile's pixels, accumulated by the tier MODE.  All threads of the CTA call
// it; shared storage is reused across calls.
template <class SH, int MODE, bool STORE_T>
__device__ __forceinline__ void backward_tile(const BwdArgs& p, const int tile, BwdSmem<SH::B, MODE>& sm,
                                              DetSmem det = DetSmem{nullptr, nullptr},
                                              const ClusterTab* ct = nullptr) {
    constexpr int B = SH::B, NT = SH::NT;
    constexpr int PPT = B / NT;
    constexpr int DG = MODE == kModeDet ? kDetGroup : B;  // entries per combine of the deterministic tier
    static_assert(MODE != GSR_REDUCE_PLAIN || PPT == 1, "the plain tier keeps one pixel per thread");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tile % p.g.gx, ty = tile / p.g.gx;
    const int ox = tx * SH::TWd, oy = ty * SH::THd;
    const uint2 rg = p.ranges[tile];
    const int nlist = (int)(rg.y - rg.x);
    const size_t HW = (size_t)p.g.W * p.g.H;

    float fpx[PPT], fpy[PPT], Tf[PPT], g0[PPT], g1[PPT], g2[PPT], T[PPT], S[PPT];
    int last[PPT];
    bool inside[PPT];
    size_t pix[PPT];
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        int lx, ly;
        SH::pixel(tid, q, lx, ly);
        const int px = ox + lx, py = oy + ly;
        inside[q] = px < p.g.W && py < p.g.H;
        fpx[q] = (float)px;
        fpy[q] = (float)py;
        pix[q] = (size_t)py * p.g.W + px;
    }
    if (STORE_T) {
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
            Tf[q] = inside[q] ? p.final_T[pix[q]] : 0.0f;
            last[q] = inside[q] ? min(max(p.n_contrib[pix[q]], 0), nlist) : 0;  // never walk past the list
        }
    } else {
        float C[PPT][3];
        walk_front<SH, false>(rg, p.point_list, p.splat2d, fpx, fpy, inside, ox, oy, sm.a, sm.b, sm.c, sm.mask, Tf,
                              last, C, p.block_mask, nullptr);
#pragma unroll
        for (int q = 0; q < PPT; ++q)
            if (!inside[q]) { Tf[q] = 0.0f; last[q] = 0; }
    }
    int mylast = 0;
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
        const bool rd = inside[q] && MODE != kModeCount;  // the count mode takes no upstream gradient
        g0[q] = rd ? p.dL_dimage[pix[q]] : 0.0f;
        g1[q] = rd ? p.dL_dimage[HW + pix[q]] : 0.0f;
        g2[q] = rd ? p.dL_dimage[2 * HW + pix[q]] : 0.0f;
        T[q] = Tf[q];
        S[q] = Tf[q] * (p.bg0 * g0[q] + p.bg1 * g1[q] + p.bg2 * g2[q]);
        mylast = max(mylast, last[q]);
    }
    __syncthreads();  // shared storage may still be read by a previous tile / the recompute walk
    if (tid == 0) sm.maxlast = 0;
    if (MODE == GSR_REDUCE_BLOCK)
        for (int i = tid; i < B * 9; i += NT) sm.acc[i] = 0.0f;
    __syncthreads();
    const int wlast = __reduce_max_sync(kFull, mylast);
    if (lane == 0) atomicMax(&sm.maxlast, wlast);
    __syncthreads();
    const int maxlast = sm.maxlast;
    const int rparam = reduce9_param(lane);
    float* __restrict__ grad = p.grad2d;
    // two pixels per thread share their column (Shape::pixel): packed state
    const float2 npy2 = make_float2(-fpy[0], -fpy[PPT - 1]);
    float2 T2 = make_float2(T[0], T[PPT - 1]), S2 = make_float2(S[0], S[PPT - 1]);
    const float2 g0_2 = make_float2(g0[0], g0[PPT - 1]), g1_2 = make_float2(g1[0], g1[PPT - 1]),
                 g2_2 = make_float2(g2[0], g2[PPT - 1]);
    unsigned long long cnt_red = 0, cnt_red4 = 0, cnt_add = 0, cnt_lane = 0, cnt_step = 0, cnt_act = 0;

    for (int top = maxlast; top > 0; top -= B) {
        const int cnt = min(B, top);
        __syncthreads();
        stage_batch<SH, true, true>(cnt, [&](int e) { return rg.x + (uint32_t)(top - 1 - e); }, p.point_list,
                                    p.splat2d, ox, oy, sm.a, sm.b, sm.c, sm.id, sm.mask, p.block_mask, nullptr);
        if (MODE == kModeDet)
            for (int e = tid; e < cnt; e += NT) det.wflags[e] = 0u;  // entries this thread staged
        __syncthreads();
        // The batch is taken in groups of DG entries: the deterministic tier
        // combines its per-warp sums after each group, the other tiers take
        // the whole batch as one group.  Each warp visits, back to front, only
        // the staged splats whose alpha >= 1/255 region touches its pixel
        // block and that lie before the warp's last contributor.
        for (int grp0 = 0; grp0 < cnt; grp0 += DG) {
            const int grp1 = min(cnt, grp0 + DG);
            for (int c0 = grp0; c0 < grp1; c0 += 32) {
                const int kq = c0 + lane;
                unsigned bits =
                    __ballot_sync(kFull, kq < grp1 && ((sm.mask[kq] >> warp) & 1u) && (top - 1 - kq < wlast));
                while (bits) {
                    const int k = c0 + __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const int pos = top - 1 - k;
                    const float4 a = sm.a[k], b = sm.b[k];
                    const float cb = sm.c[k];
                    // every lane runs the gradient chain for every pixel slot; an
                    // inactive pair enters it with alpha = G = 0, which leaves T and
                    // S unchanged (1 / (1 - 0) is exactly 1 after the Newton step)
                    // and adds only zeros
                    float v[9];
                    bool any = false;
                    if constexpr (PPT == 2) {
                        SplatEval2 e;
                        bool act0, act1;
                        eval_splat2_all(a.x, a.y, a.z, a.w, b.x, b.y, fpx[0], npy2, e, act0, act1);
                        act0 = act0 && pos < last[0];
                        act1 = act1 && pos < last[1];
                        pair_grads2(e, act0, act1, a, b, cb, g0_2, g1_2, g2_2, T2, S2, v);
                        any = act0 || act1;
                    } else {
#pragma unroll
                        for (int q = 0; q < PPT; ++q) {
                            SplatEval e;
                            const bool act =
                                eval_splat_all(a.x, a.y, a.z, a.w, b.x, b.y, fpx[q], fpy[q], e) && (pos < last[q]);
                            e.alpha = act ? e.alpha : 0.0f;
                            e.G = act ? e.G : 0.0f;
                            if (q == 0) pair_grads<true>(e, a, b, cb, g0[q], g1[q], g2[q], T[q], S[q], v);
                            else pair_grads<false>(e, a, b, cb, g0[q], g1[q], g2[q], T[q], S[q], v);
                            any |= act;
                        }
                    }
                    if (MODE == kModeCount) {
                        const unsigned m = __ballot_sync(kFull, any);
                        const unsigned long long a = (unsigned long long)__popc(m);
                        if (lane == 0) atomicAdd(&p.counts[6 + a], 1ull);
                        cnt_step += 1;
                        if (a == 0) continue;
                        cnt_act += 1;
                        if (p.count_tier == GSR_REDUCE_PLAIN) {  // 9 scalar atomics per active lane
                            cnt_red += 9; cnt_add += 9 * a; cnt_lane += 9 * a;
                        } else if (p.count_tier == GSR_REDUCE_WARP || (int)a >= p.threshold) {  // one 9-lane red
                            cnt_red += 1; cnt_add += 9; cnt_lane += 9;
                        } else {  // two v4 reds and one scalar per active lane
                            cnt_red += 1; cnt_red4 += 2; cnt_add += 9 * a; cnt_lane += 3 * a;
                        }
                        continue;
                    }
                    float* rec = grad + (size_t)sm.id[k] * GSR_REC;
                    if (MODE == kModeDet) {
                        if (__ballot_sync(kFull, any) == 0u) continue;
                        const float z = reduce9(v, lane);
                        if (rparam < 9) det.part[(warp * DG + (k - grp0)) * 9 + rparam] = z;
                        if (lane == 0) atomicOr(&det.wflags[k], 1u << warp);
                    } else if (MODE == GSR_REDUCE_PLAIN) {
                        if (any) {
#pragma unroll
                            for (int i = 0; i < 9; ++i) atomicAdd(rec + i, v[i]);
                        }
                    } else {
                        const unsigned m = __ballot_sync(kFull, any);
                        if (m == 0u) continue;
                        const bool dense = (MODE == GSR_REDUCE_WARP) || (__popc(m) >= p.threshold);
                        if (dense) {
                            const float z = reduce9(v, lane);
                            if (MODE == kModeCluster) {
                                uint32_t owner = 0;
                                int slot = -1;
                                if (lane == 0) slot = cluster_slot(*ct, sm.id[k], owner);
                                slot = __shfl_sync(kFull, slot, 0);
                                owner = __shfl_sync(kFull, owner, 0);
                                if (rparam < 9) {
                                    if (slot >= 0) {
                                        const uint32_t la = ct->val_base + 4u * (uint32_t)(slot * 9 + rparam);
                                        dsm_red_add(cluster_map(la, owner), z);
                                    } else {
                                        red_add(rec + rparam, z);
                                    }
                                }
                            } else if (rparam < 9) {
                                if (MODE == GSR_REDUCE_BLOCK) atomicAdd(&sm.acc[k * 9 + rparam], z);
                                else red_add(rec + rparam, z);
                            }
                        } else if (any) {
                            if (MODE == GSR_REDUCE_BLOCK) {
#pragma unroll
                                for (int i = 0; i < 9; ++i) atomicAdd(&sm.acc[k * 9 + i], v[i]);
                            } else {  // the 16-byte-aligned record takes two vector reds and one scalar
                                red_add_v4(rec, v[0], v[1], v[2], v[3]);
                                red_add_v4(rec + 4, v[4], v[5], v[6], v[7]);
                                red_add(rec + 8, v[8]);
                            }
                        }
                    }
                }
            }
            if (MODE == kModeDet) {
                // warp partials combined in warp order: a fixed summation order
                __syncthreads();
                for (int k = grp0 + tid; k < grp1; k += NT) {
                    const unsigned fl = det.wflags[k];
                    if (fl == 0u) continue;  // the slot keeps the zeros it was cleared to
                    float* dst = p.partial + 9 * (size_t)entry_slot(p, sm.id[k], sm.a[k].x, sm.a[k].y, tile);
#pragma unroll
                    for (int q = 0; q < 9; ++q) {
                        float sum = 0.0f;
#pragma unroll
                        for (int w = 0; w < SH::NW; ++w)
                            if ((fl >> w) & 1u) sum += det.part[(w * DG + (k - grp0)) * 9 + q];
                        dst[q] = sum;
                    }
                }
                if (grp1 < cnt) __syncthreads();  // the next group reuses the partial sums' storage
            }
        }
        if (MODE == GSR_REDUCE_BLOCK) {
            __syncthreads();
            for (int i = tid; i < cnt * 9; i += NT) {
                const float val = sm.acc[i];
                if (val != 0.0f) {
                    const int k = i / 9;
                    red_add(grad + (size_t)sm.id[k] * GSR_REC + (i - 9 * k), val);
                    sm.acc[i] = 0.0f;
                }
            }
        }
    }
    if (MODE == kModeCount && lane == 0 && cnt_step) {
        atomicAdd(&p.counts[0], cnt_red);
        atomicAdd(&p.counts[1], cnt_red4);
        atomicAdd(&p.counts[2], cnt_add);
        atomicAdd(&p.counts[3], cnt_lane);
        atomicAdd(&p.counts[4], cnt_step);
        atomicAdd(&p.counts[5], cnt_act);
    }
}

}  // namespace gsr
