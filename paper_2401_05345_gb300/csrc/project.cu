// Projection of 3D Gaussians to 2D splats (forward) and the chain rule back
// to the 3D parameters (backward projection).  One thread per Gaussian.
#include <math.h>

#include "gsr_internal.cuh"

namespace gsr {
namespace {

struct Cam {
    float R[9], t[3];
    float fx, fy, cx, cy, limx, limy, znear;
    float campos[3];
    int W, H;
};

Cam make_cam(const gsr_camera& c) {
    Cam k;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) k.R[3 * i + j] = c.view[4 * i + j];
        k.t[i] = c.view[4 * i + 3];
        k.campos[i] = c.campos[i];
    }
    k.fx = c.fx; k.fy = c.fy; k.cx = c.cx; k.cy = c.cy;
    k.limx = kFrustum * c.tan_fovx;
    k.limy = kFrustum * c.tan_fovy;
    k.znear = c.znear;
    k.W = c.width; k.H = c.height;
    return k;
}

// Real SH basis up to degree 3 (3DGS sign convention), orthonormal on the
// sphere; Y[k] for k < (deg+1)^2.
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
    const float C0 = 0.28209479177387814f;
    const float C1 = 0.4886025119029199f;
    const float C2a = 1.0925484305920792f, C2b = 0.31539156525252005f, C2c = 0.5462742152960396f;
    const float C3a = 0.5900435899266435f, C3b = 2.890611442640554f, C3c = 0.4570457994644658f;
    const float C3d = 0.3731763325901154f, C3e = 1.445305721320277f;
    Y[0] = C0;
    if (deg < 1) return;
    Y[1] = -C1 * y; Y[2] = C1 * z; Y[3] = -C1 * x;
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = C2a * x * y;
    Y[5] = -C2a * y * z;
    Y[6] = C2b * (2.f * zz - xx - yy);
    Y[7] = -C2a * x * z;
    Y[8] = C2c * (xx - yy);
    if (deg < 3) return;
    Y[9] = -C3a * y * (3.f * xx - yy);
    Y[10] = C3b * x * y * z;
    Y[11] = -C3c * y * (4.f * zz - xx - yy);
    Y[12] = C3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
    Y[13] = -C3c * x * (4.f * zz - xx - yy);
    Y[14] = C3e * z * (xx - yy);
    Y[15] = -C3a * x * (xx - 3.f * yy);
}

// Gradient of sum_k c[k] Y_k(x,y,z) w.r.t. (x,y,z) treated as free variables.
__device__ __forceinline__ void sh_basis_vjp(int deg, float x, float y, float z, const float* c,
                                             float& gx, float& gy, float& gz) {
    const float C1 = 0.4886025119029199f;
    const float C2a = 1.0925484305920792f, C2b = 0.31539156525252005f, C2c = 0.5462742152960396f;
    const float C3a = 0.5900435899266435f, C3b = 2.890611442640554f, C3c = 0.4570457994644658f;
    const float C3d = 0.3731763325901154f, C3e = 1.445305721320277f;
    gx = gy = gz = 0.f;
    if (deg < 1) return;
    gy += -C1 * c[1]; gz += C1 * c[2]; gx += -C1 * c[3];
    if (deg < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    gx += C2a * y * c[4]; gy += C2a * x * c[4];
    gy += -C2a * z * c[5]; gz += -C2a * y * c[5];
    gx += -2.f * C2b * x * c[6]; gy += -2.f * C2b * y * c[6]; gz += 4.f * C2b * z * c[6];
    gx += -C2a * z * c[7]; gz += -C2a * x * c[7];
    gx += 2.f * C2c * x * c[8]; gy += -2.f * C2c * y * c[8];
    if (deg < 3) return;
    gx += -C3a * 6.f * x * y * c[9]; gy += -C3a * (3.f * xx - 3.f * yy) * c[9];
    gx += C3b * y * z * c[10]; gy += C3b * x * z * c[10]; gz += C3b * x * y * c[10];
    gx += C3c * 2.f * x * y * c[11]; gy += -C3c * (4.f * zz - xx - 3.f * yy) * c[11];
    gz += -C3c * 8.f * y * z * c[11];
    gx += -C3d * 6.f * x * z * c[12]; gy += -C3d * 6.f * y * z * c[12];
    gz += C3d * (6.f * zz - 3.f * xx - 3.f * yy) * c[12];
    gx += -C3c * (4.f * zz - 3.f * xx - yy) * c[13]; gy += C3c * 2.f * x * y * c[13];
    gz += -C3c * 8.f * x * z * c[13];
    gx += C3e * 2.f * x * z * c[14]; gy += -C3e * 2.f * y * z * c[14]; gz += C3e * (xx - yy) * c[14];
    gx += -C3a * (3.f * xx - 3.f * yy) * c[15]; gy += C3a * 6.f * x * y * c[15];
}

// Feature rows of a chunk of CH Gaussians staged through shared memory:
// global rows of NF floats are read (and written back) with coalesced
// 16-byte accesses when VEC, and kept in shared memory with an odd row
// stride NF + 1 so that each thread's own row is read without bank conflicts.
template <int NF>
__device__ __forceinline__ int srow(int f) { return (f / NF) * (NF + 1) + f % NF; }

template <int NF, int CH, bool VEC>
__device__ __forceinline__ void stage_rows_in(const float* __restrict__ g, int rows, float* s) {
    if constexpr (VEC && NF % 4 == 0) {
        if (rows == CH) {  // a full chunk: every 16-byte load in flight at once
            constexpr int Q = NF / 4;
            const float4* g4 = reinterpret_cast<const float4*>(g);
            float4 x[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) x[q] = g4[threadIdx.x + q * CH];
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const int f = 4 * (threadIdx.x + q * CH);
                s[srow<NF>(f)] = x[q].x;
                s[srow<NF>(f + 1)] = x[q].y;
                s[srow<NF>(f + 2)] = x[q].z;
                s[srow<NF>(f + 3)] = x[q].w;
            }
            return;
        }
    }
    const int total = rows * NF;
    int f0 = 0;
    if (VEC) {
        const float4* g4 = reinterpret_cast<const float4*>(g);
        const int n4 = total >> 2;
        for (int t = threadIdx.x; t < n4; t += CH) {
            const float4 x = g4[t];
            const int f = 4 * t;
            s[srow<NF>(f)] = x.x;
            s[srow<NF>(f + 1)] = x.y;
            s[srow<NF>(f + 2)] = x.z;
            s[srow<NF>(f + 3)] = x.w;
        }
        f0 = n4 << 2;
    }
    for (int f = f0 + threadIdx.x; f < total; f += CH) s[srow<NF>(f)] = g[f];
}

template <int NF, int CH, bool VEC>
__device__ __forceinline__ void stage_rows_add_out(float* __restrict__ g, int rows, const float* s) {
    const int total = rows * NF;
    int f0 = 0;
    if (VEC) {
        float4* g4 = reinterpret_cast<float4*>(g);
        const int n4 = total >> 2;
        for (int t = threadIdx.x; t < n4; t += CH) {
            float4 x = g4[t];
            const int f = 4 * t;
            x.x += s[srow<NF>(f)];
            x.y += s[srow<NF>(f + 1)];
            x.z += s[srow<NF>(f + 2)];
            x.w += s[srow<NF>(f + 3)];
            g4[t] = x;
        }
        f0 = n4 << 2;
    }
    for (int f = f0 + threadIdx.x; f < total; f += CH) g[f] += s[srow<NF>(f)];
}

// Writes the staged rows back: g += s (ACC) or g = s.
template <int NF, int CH, bool VEC, bool ACC>
__device__ __forceinline__ void stage_rows_out(float* __restrict__ g, int rows, const float* s) {
    if (ACC) {
        stage_rows_add_out<NF, CH, VEC>(g, rows, s);
        return;
    }
    const int total = rows * NF;
    int f0 = 0;
    if (VEC) {
        float4* g4 = reinterpret_cast<float4*>(g);
        const int n4 = total >> 2;
        for (int t = threadIdx.x; t < n4; t += CH) {
            const int f = 4 * t;
            g4[t] = make_float4(s[srow<NF>(f)], s[srow<NF>(f + 1)], s[srow<NF>(f + 2)], s[srow<NF>(f + 3)]);
        }
        f0 = n4 << 2;
    }
    for (int f = f0 + threadIdx.x; f < total; f += CH) g[f] = s[srow<NF>(f)];
}

// out += v (ACC) or out = v.
template <bool ACC>
__device__ __forceinline__ void put(float& out, float v) {
    if (ACC) out += v;
    else out = v;
}

constexpr int kChunk = 128;  // Gaussians per CTA of the projection kernels

// Forward quantities of one Gaussian, kept for the backward projection.
struct Proj {
    float p[3];          // camera-space mean
    float qn[4], qinv;   // normalised quaternion, 1/|q|
    float R[9];          // rotation
    float M[9];          // R diag(s)
    float S3[6];         // 3D covariance (xx, xy, xz, yy, yz, zz)
    float tx, ty;        // clamped x/z, y/z
    bool clx, cly;
    float T[6];          // J W (2x3)
    float a, b, c, det;  // dilated 2D covariance [[a,b],[b,c]]
    float u, v;
};

// Returns false if culled behind the near plane or degenerate.
__device__ __forceinline__ bool project(const Cam& k, const float* mean, const float* scale,
                                        const float* quat, Proj& P) {
    const float mx = mean[0], my = mean[1], mz = mean[2];
    for (int i = 0; i < 3; ++i)
        P.p[i] = fmaf(k.R[3 * i], mx, fmaf(k.R[3 * i + 1], my, fmaf(k.R[3 * i + 2], mz, k.t[i])));
    if (!(P.p[2] > k.znear)) return false;
    float q0 = quat[0], q1 = quat[1], q2 = quat[2], q3 = quat[3];
    float qq = q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3;
    P.qinv = 1.0f / sqrtf(qq);
    float w = q0 * P.qinv, x = q1 * P.qinv, y = q2 * P.qinv, z = q3 * P.qinv;
    P.qn[0] = w; P.qn[1] = x; P.qn[2] = y; P.qn[3] = z;
    float* R = P.R;
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) P.M[3 * i + j] = R[3 * i + j] * scale[j];
    const float* M = P.M;
    auto dot3 = [](const float* a, const float* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
    P.S3[0] = dot3(M, M);         P.S3[1] = dot3(M, M + 3);     P.S3[2] = dot3(M, M + 6);
    P.S3[3] = dot3(M + 3, M + 3); P.S3[4] = dot3(M + 3, M + 6); P.S3[5] = dot3(M + 6, M + 6);

    const float pz = P.p[2];
    const float iz = 1.0f / pz;
    float xz = P.p[0] * iz, yz = P.p[1] * iz;
    P.clx = (xz < -k.limx) || (xz > k.limx);
    P.cly = (yz < -k.limy) || (yz > k.limy);
    P.tx = fminf(k.limx, fmaxf(-k.limx, xz));
    P.ty = fminf(k.limy, fmaxf(-k.limy, yz));
    float J00 = k.fx * iz, J02 = -k.fx * P.tx * iz, J11 = k.fy * iz, J12 = -k.fy * P.ty * iz;
    for (int j = 0; j < 3; ++j) {
        P.T[j] = J00 * k.R[j] + J02 * k.R[6 + j];
        P.T[3 + j] = J11 * k.R[3 + j] + J12 * k.R[6 + j];
    }
    // Sigma2 = T S3 T^T
    const float* S = P.S3;
    float Sm[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
    float t0[3], t1[3];
    for (int j = 0; j < 3; ++j) {
        t0[j] = P.T[0] * Sm[j] + P.T[1] * Sm[3 + j] + P.T[2] * Sm[6 + j];
        t1[j] = P.T[3] * Sm[j] + P.T[4] * Sm[3 + j] + P.T[5] * Sm[6 + j];
    }
    P.a = t0[0] * P.T[0] + t0[1] * P.T[1] + t0[2] * P.T[2] + kDilation;
    P.b = t0[0] * P.T[3] + t0[1] * P.T[4] + t0[2] * P.T[5];
    P.c = t1[0] * P.T[3] + t1[1] * P.T[4] + t1[2] * P.T[5] + kDilation;
    P.det = P.a * P.c - P.b * P.b;
    if (!(P.det > 0.0f)) return false;
    P.u = fmaf(k.fx * P.p[0], iz, k.cx);
    P.v = fmaf(k.fy * P.p[1], iz, k.cy);
    return true;
}

// One 32-byte load of read-only data (p 32-byte aligned) into two float4s.
__device__ __forceinline__ void ld_nc_v8(const float* p, float4& a, float4& b) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// Load widths the caller's alignment allows (uniform over the launch).
constexpr int kWideFeat = 1;  // feature rows 32-byte aligned (base 32-byte aligned, rows a multiple of 32 B)
constexpr int kWideQuat = 2;  // quaternion rows 16-byte aligned

template <int DEG, bool VEC>
__global__ void __launch_bounds__(kChunk)
preprocess_kernel(int n, const float* __restrict__ mean, const float* __restrict__ scale,
                  const float* __restrict__ quat, const float* __restrict__ opacity,
                  const float* __restrict__ feat, Cam k, int gx, int gy, int tw_log2, int th_log2,
                  float* __restrict__ splat2d, int* __restrict__ radius, float* __restrict__ gzero,
                  int wide) {
    constexpr int K = DEG < 0 ? 1 : (DEG + 1) * (DEG + 1);
    constexpr int NF = 3 * K;
    // rows of whole 16-byte words: every thread loads its own row into
    // registers (no staging, no barrier), 32 bytes a load where the rows
    // allow it
    constexpr bool DIRECT = VEC && DEG >= 1 && NF % 4 == 0;
    __shared__ float s_f[DEG < 0 || DIRECT ? 1 : kChunk * (NF + 1)];
    const int base = blockIdx.x * kChunk;
    const int i = base + threadIdx.x;
    float4 fr[DIRECT ? NF / 4 : 1];
    if constexpr (DIRECT) {
        if (i < n) {
            const float* row = feat + (size_t)i * NF;
            if (NF % 8 == 0 && (wide & kWideFeat)) {
#pragma unroll
                for (int q = 0; q < NF / 8; ++q) ld_nc_v8(row + 8 * q, fr[2 * q], fr[2 * q + 1]);
            } else {
                const float4* g4 = reinterpret_cast<const float4*>(row);
#pragma unroll
                for (int q = 0; q < NF / 4; ++q) fr[q] = g4[q];
            }
        }
    }
    // this Gaussian's other inputs are requested before the feature staging
    // (with rows in registers: right after the row's loads), so all of
    // their latencies overlap
    float mv[3] = {0.f, 0.f, 0.f}, sv[3] = {0.f, 0.f, 0.f}, qv[4] = {1.f, 0.f, 0.f, 0.f}, op = 0.f;
    if (i < n) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            mv[j] = mean[3 * (size_t)i + j];
            sv[j] = scale[3 * (size_t)i + j];
        }
        if (wide & kWideQuat) {
            const float4 q4 = *reinterpret_cast<const float4*>(quat + 4 * (size_t)i);
            qv[0] = q4.x;
            qv[1] = q4.y;
            qv[2] = q4.z;
            qv[3] = q4.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) qv[j] = quat[4 * (size_t)i + j];
        }
        op = opacity[i];
    }
    if constexpr (DEG >= 0 && !DIRECT) {
        stage_rows_in<NF, kChunk, VEC>(feat + (size_t)base * NF, min(kChunk, n - base), s_f);
        __syncthreads();
    }
    if (i >= n) return;
    float4* rec = reinterpret_cast<float4*>(splat2d + (size_t)i * GSR_REC);
    if (gzero) {
        float4* gz = reinterpret_cast<float4*>(gzero + (size_t)i * GSR_REC);
        gz[0] = gz[1] = gz[2] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    Proj P;
    int r = 0;
    bool ok = project(k, mv, sv, qv, P);
    if (ok) {
        float mid = 0.5f * (P.a + P.c);
        float disc = fmaxf(kLambdaFloor, mid * mid - P.det);
        float lam = mid + sqrtf(disc);
        r = (int)ceilf(3.0f * sqrtf(lam));
        int x0, x1, y0, y1;
        float uc = fminf(fmaxf(P.u, -1e8f), 1e8f), vc = fminf(fmaxf(P.v, -1e8f), 1e8f);
        tile_rect(uc, vc, r, gx, gy, tw_log2, th_log2, x0, x1, y0, y1);
        if ((x1 - x0) * (y1 - y0) <= 0) ok = false;
    }
    if (!ok) {
        radius[i] = 0;
        rec[0] = rec[1] = rec[2] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    float idet = 1.0f / P.det;
    float rgb[3];
    if constexpr (DEG < 0) {
        for (int ch = 0; ch < 3; ++ch) rgb[ch] = feat[3 * (size_t)i + ch];
    } else {
        float dx = mv[0] - k.campos[0], dy = mv[1] - k.campos[1], dz = mv[2] - k.campos[2];
        float il = 1.0f / sqrtf(dx * dx + dy * dy + dz * dz);
        float Y[16];
        sh_basis(DEG, dx * il, dy * il, dz * il, Y);
        const float* f = s_f + threadIdx.x * (NF + 1);
        // feature x of the row (x a compile-time index after unrolling)
        auto F = [&](int x) -> float {
            if constexpr (DIRECT) {
                const float4 w = fr[x >> 2];
                return (x & 3) == 0 ? w.x : (x & 3) == 1 ? w.y : (x & 3) == 2 ? w.z : w.w;
            } else {
                return f[x];
            }
        };
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            s0 = fmaf(Y[j], F(3 * j), s0);
            s1 = fmaf(Y[j], F(3 * j + 1), s1);
            s2 = fmaf(Y[j], F(3 * j + 2), s2);
        }
        rgb[0] = fmaxf(s0 + 0.5f, 0.f);
        rgb[1] = fmaxf(s1 + 0.5f, 0.f);
        rgb[2] = fmaxf(s2 + 0.5f, 0.f);
    }
    radius[i] = r;
    rec[0] = make_float4(P.u, P.v, P.c * idet, -P.b * idet);
    rec[1] = make_float4(P.a * idet, op, rgb[0], rgb[1]);
    rec[2] = make_float4(rgb[2], P.p[2], 0.f, 0.f);
}

// ACC: gradients are added to the outputs; otherwise every output element of
// every Gaussian is written (zero for culled Gaussians).
// Six CTAs per SM (at most 80 registers): the kernel is bound by memory
// latency, so resident warps matter more than registers.
template <int DEG, bool VEC, bool ACC>
__global__ void __launch_bounds__(kChunk, 6)
backproject_kernel(int n, const float* __restrict__ mean, const float* __restrict__ scale,
                   const float* __restrict__ quat, const float* __restrict__ feat, Cam k,
                   const int* __restrict__ radius, const float* __restrict__ grad2d,
                   float* __restrict__ dmean, float* __restrict__ dscale, float* __restrict__ dquat,
                   float* __restrict__ dopacity, float* __restrict__ dfeat) {
    constexpr int K = DEG < 0 ? 1 : (DEG + 1) * (DEG + 1);
    constexpr int NF = 3 * K;
    __shared__ float s_f[DEG < 0 ? 1 : kChunk * (NF + 1)];
    const int base = blockIdx.x * kChunk;
    const int rows = min(kChunk, n - base);
    const int i = base + threadIdx.x;
    const bool valid = i < n && radius[i] > 0;
    float dm[3] = {0.f, 0.f, 0.f};
    float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), gb = ga, gc = ga;
    // this Gaussian's inputs are requested before the feature staging, so
    // their latency overlaps it
    float mv[3] = {0.f, 0.f, 0.f}, sv[3] = {0.f, 0.f, 0.f}, qv[4] = {1.f, 0.f, 0.f, 0.f};
    if (valid) {
        const float4* g4 = reinterpret_cast<const float4*>(grad2d + (size_t)i * GSR_REC);
        ga = g4[0];
        gb = g4[1];
        gc = g4[2];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            mv[j] = mean[3 * (size_t)i + j];
            sv[j] = scale[3 * (size_t)i + j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) qv[j] = quat[4 * (size_t)i + j];
    }
    float gcol[3] = {gb.z, gb.w, gc.x};

    // colour: SH basis along the viewing direction, clamp at 0
    if constexpr (DEG < 0) {
        if (valid)
            for (int ch = 0; ch < 3; ++ch) put<ACC>(dfeat[3 * (size_t)i + ch], gcol[ch]);
        else if (!ACC && i < n)
            for (int ch = 0; ch < 3; ++ch) dfeat[3 * (size_t)i + ch] = 0.f;
    } else {
        stage_rows_in<NF, kChunk, VEC>(feat + (size_t)base * NF, rows, s_f);
        __syncthreads();
        float* f = s_f + threadIdx.x * (NF + 1);
        if (valid) {
            float dx = mv[0] - k.campos[0], dy = mv[1] - k.campos[1], dz = mv[2] - k.campos[2];
            float len = sqrtf(dx * dx + dy * dy + dz * dz);
            float il = 1.0f / len;
            float x = dx * il, y = dy * il, z = dz * il;
            float Y[16];
            sh_basis(DEG, x, y, z, Y);
            float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
            for (int j = 0; j < K; ++j)
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) raw[ch] = fmaf(Y[j], f[3 * j + ch], raw[ch]);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) if (raw[ch] < 0.f) gcol[ch] = 0.f;
            float cw[16];
#pragma unroll
            for (int j = 0; j < K; ++j) {
                cw[j] = f[3 * j] * gcol[0] + f[3 * j + 1] * gcol[1] + f[3 * j + 2] * gcol[2];
                // this thread's row now receives its feature gradient
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) f[3 * j + ch] = Y[j] * gcol[ch];
            }
            float ddx, ddy, ddz;
            sh_basis_vjp(DEG, x, y, z, cw, ddx, ddy, ddz);
            float dot = x * ddx + y * ddy + z * ddz;
            dm[0] += (ddx - x * dot) * il;
            dm[1] += (ddy - y * dot) * il;
            dm[2] += (ddz - z * dot) * il;
        } else if (threadIdx.x < rows) {
#pragma unroll
            for (int j = 0; j < NF; ++j) f[j] = 0.f;
        }
        __syncthreads();
        stage_rows_out<NF, kChunk, VEC, ACC>(dfeat + (size_t)base * NF, rows, s_f);
    }
    Proj P;
    const float* s = sv;
    if (!valid || !project(k, mv, sv, qv, P)) {
        if (!ACC && i < n) {  // the outputs of a culled Gaussian are zero
            dopacity[i] = 0.f;
            for (int j = 0; j < 3; ++j) dmean[3 * (size_t)i + j] = dscale[3 * (size_t)i + j] = 0.f;
            for (int j = 0; j < 4; ++j) dquat[4 * (size_t)i + j] = 0.f;
        }
        return;
    }
    const float gu = ga.x, gv = ga.y, gA = ga.z, gB = ga.w, gC = gb.x, go = gb.y;
    put<ACC>(dopacity[i], go);

    // conic (A,B,C) = inverse of [[a,b],[b,c]]
    const float a = P.a, b = P.b, c = P.c;
    float id = 1.0f / P.det;
    float id2 = id * id;
    float da = (-c * c * gA + b * c * gB - b * b * gC) * id2;
    float db = (2.f * b * c * gA - (a * c + b * b) * gB + 2.f * a * b * gC) * id2;
    float dc = (-b * b * gA + a * b * gB - a * a * gC) * id2;
    const float G00 = da, G01 = 0.5f * db, G11 = dc;

    // Sigma2 = T S3 T^T
    const float* T = P.T;
    const float* S = P.S3;
    float Sm[9] = {S[0], S[1], S[2], S[1], S[3], S[4], S[2], S[4], S[5]};
    float dS3[9];
    for (int ii = 0; ii < 3; ++ii)
        for (int jj = 0; jj < 3; ++jj)
            dS3[3 * ii + jj] = T[ii] * (G00 * T[jj] + G01 * T[3 + jj]) +
                               T[3 + ii] * (G01 * T[jj] + G11 * T[3 + jj]);
    // dL/dT = 2 G2 T S3
    float TS0[3], TS1[3];
    for (int j = 0; j < 3; ++j) {
        TS0[j] = T[0] * Sm[j] + T[1] * Sm[3 + j] + T[2] * Sm[6 + j];
        TS1[j] = T[3] * Sm[j] + T[4] * Sm[3 + j] + T[5] * Sm[6 + j];
    }
    float dT[6];
    for (int j = 0; j < 3; ++j) {
        dT[j] = 2.f * (G00 * TS0[j] + G01 * TS1[j]);
        dT[3 + j] = 2.f * (G01 * TS0[j] + G11 * TS1[j]);
    }
    // S3 = M M^T: dL/dM = 2 dS3 M; M = R diag(s)
    float dR[9];
    float* ds = dscale + 3 * (size_t)i;
    for (int j = 0; j < 3; ++j) {
        float acc = 0.f;
        for (int ii = 0; ii < 3; ++ii) {
            float dMij = 2.f * (dS3[3 * ii] * P.M[j] + dS3[3 * ii + 1] * P.M[3 + j] + dS3[3 * ii + 2] * P.M[6 + j]);
            acc += dMij * P.R[3 * ii + j];
            dR[3 * ii + j] = dMij * s[j];
        }
        put<ACC>(ds[j], acc);
    }
    // R(q) with q normalised, then through the normalisation
    const float w = P.qn[0], x = P.qn[1], y = P.qn[2], z = P.qn[3];
    float dq[4];
    dq[0] = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    dq[1] = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] + w * dR[7] - 2.f * x * dR[8]);
    dq[2] = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] + z * dR[7] - 2.f * y * dR[8]);
    dq[3] = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] + y * dR[5] + x * dR[6] + y * dR[7]);
    float qd = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
    float* dqo = dquat + 4 * (size_t)i;
    for (int j = 0; j < 4; ++j) put<ACC>(dqo[j], (dq[j] - P.qn[j] * qd) * P.qinv);

    // T = J W: dL/dJ = dT W^T (only J00, J02, J11, J12 are non-zero)
    float dJ00 = dT[0] * k.R[0] + dT[1] * k.R[1] + dT[2] * k.R[2];
    float dJ02 = dT[0] * k.R[6] + dT[1] * k.R[7] + dT[2] * k.R[8];
    float dJ11 = dT[3] * k.R[3] + dT[4] * k.R[4] + dT[5] * k.R[5];
    float dJ12 = dT[3] * k.R[6] + dT[4] * k.R[7] + dT[5] * k.R[8];
    const float pz = P.p[2], iz = 1.0f / pz, iz2 = iz * iz;
    float dJ02_dx = P.clx ? 0.f : -k.fx * iz2;
    float dJ02_dz = k.fx * P.tx * iz2 * (P.clx ? 1.f : 2.f);
    float dJ12_dy = P.cly ? 0.f : -k.fy * iz2;
    float dJ12_dz = k.fy * P.ty * iz2 * (P.cly ? 1.f : 2.f);
    float dp0 = gu * k.fx * iz + dJ02 * dJ02_dx;
    float dp1 = gv * k.fy * iz + dJ12 * dJ12_dy;
    float dp2 = -(gu * k.fx * P.p[0] + gv * k.fy * P.p[1]) * iz2 - dJ00 * k.fx * iz2 - dJ11 * k.fy * iz2 +
                dJ02 * dJ02_dz + dJ12 * dJ12_dz;
    float* dmo = dmean + 3 * (size_t)i;
    for (int j = 0; j < 3; ++j)
        put<ACC>(dmo[j], dm[j] + k.R[j] * dp0 + k.R[3 + j] * dp1 + k.R[6 + j] * dp2);
}

bool tiles_ok(int tw, int th) { return pow2_in(tw, 8, 32) && pow2_in(th, 8, 32) && tw * th <= 512; }
int ilog2(int x) { int l = 0; while ((1 << l) < x) ++l; return l; }

}  // namespace
}  // namespace gsr

using namespace gsr;

extern "C" int gsr_preprocess(int32_t n, int32_t sh_degree, const float* mean, const float* scale,
                              const float* quat, const float* opacity, const float* feat,
                              const gsr_camera* cam, int32_t tile_w, int32_t tile_h, float* splat2d,
                              int32_t* radius, float* grad2d_to_zero, gsr_stream_t stream) {
    if (n < 0 || sh_degree < -1 || sh_degree > 3 || !cam || !tiles_ok(tile_w, tile_h)) return GSR_EINVAL;
    if (n == 0) return GSR_OK;
    if (!mean || !scale || !quat || !opacity || !feat || !splat2d || !radius) return GSR_EINVAL;
    if (!aligned16(splat2d) || (grad2d_to_zero && !aligned16(grad2d_to_zero))) return GSR_EINVAL;
    if (cam->width <= 0 || cam->height <= 0) return GSR_EINVAL;
    Cam k = make_cam(*cam);
    int gx = (cam->width + tile_w - 1) / tile_w, gy = (cam->height + tile_h - 1) / tile_h;
    const int blocks = (n + kChunk - 1) / kChunk;
    cudaStream_t st = (cudaStream_t)stream;
    const int twl = ilog2(tile_w), thl = ilog2(tile_h);
    const bool vec = aligned16(feat);
    const int wide = (((uintptr_t)feat & 31u) == 0 ? kWideFeat : 0) | (aligned16(quat) ? kWideQuat : 0);
#define GSR_PRE(D)                                                                                          \
    do {                                                                                                    \
        if (vec) preprocess_kernel<D, true><<<blocks, kChunk, 0, st>>>(n, mean, scale, quat, opacity, feat, k, \
                                                                    gx, gy, twl, thl, splat2d, radius,      \
                                                                    grad2d_to_zero, wide);                  \
        else preprocess_kernel<D, false><<<blocks, kChunk, 0, st>>>(n, mean, scale, quat, opacity, feat, k,   \
                                                                 gx, gy, twl, thl, splat2d, radius,         \
                                                                 grad2d_to_zero, wide);                     \
    } while (0)
    switch (sh_degree) {
        case -1: GSR_PRE(-1); break;
        case 0: GSR_PRE(0); break;
        case 1: GSR_PRE(1); break;
        case 2: GSR_PRE(2); break;
        default: GSR_PRE(3); break;
    }
#undef GSR_PRE
    return check_launch();
}

template <bool ACC>
int backward_project_impl(int32_t n, int32_t sh_degree, const float* mean, const float* scale, const float* quat,
                          const float* feat, const gsr_camera* cam, const int32_t* radius, const float* grad2d,
                          float* dmean, float* dscale, float* dquat, float* dopacity, float* dfeat,
                          gsr_stream_t stream) {
    if (n < 0 || sh_degree < -1 || sh_degree > 3 || !cam) return GSR_EINVAL;
    if (n == 0) return GSR_OK;
    if (!mean || !scale || !quat || !feat || !radius || !grad2d || !dmean || !dscale || !dquat ||
        !dopacity || !dfeat)
        return GSR_EINVAL;
    if (!aligned16(grad2d)) return GSR_EINVAL;
    Cam k = make_cam(*cam);
    const int blocks = (n + kChunk - 1) / kChunk;
    cudaStream_t st = (cudaStream_t)stream;
    const bool vec = aligned16(feat) && aligned16(dfeat);
#define GSR_BP(D)                                                                                                  \
    do {                                                                                                           \
        if (vec) backproject_kernel<D, true, ACC><<<blocks, kChunk, 0, st>>>(n, mean, scale, quat, feat, k, radius, \
                                                                           grad2d, dmean, dscale, dquat,            \
                                                                           dopacity, dfeat);                        \
        else backproject_kernel<D, false, ACC><<<blocks, kChunk, 0, st>>>(n, mean, scale, quat, feat, k, radius,   \
                                                                        grad2d, dmean, dscale, dquat, dopacity,    \
                                                                        dfeat);                                    \
    } while (0)
    switch (sh_degree) {
        case -1: GSR_BP(-1); break;
        case 0: GSR_BP(0); break;
        case 1: GSR_BP(1); break;
        case 2: GSR_BP(2); break;
        default: GSR_BP(3); break;
    }
#undef GSR_BP
    return check_launch();
}

extern "C" int gsr_backward_project(int32_t n, int32_t sh_degree, const float* mean, const float* scale,
                                    const float* quat, const float* opacity, const float* feat,
                                    const gsr_camera* cam, const int32_t* radius, const float* grad2d,
                                    float* dmean, float* dscale, float* dquat, float* dopacity,
                                    float* dfeat, gsr_stream_t stream) {
    (void)opacity;
    return backward_project_impl<true>(n, sh_degree, mean, scale, quat, feat, cam, radius, grad2d, dmean, dscale,
                                       dquat, dopacity, dfeat, stream);
}

extern "C" int gsr_backward_project_store(int32_t n, int32_t sh_degree, const float* mean, const float* scale,
                                          const float* quat, const float* opacity, const float* feat,
                                          const gsr_camera* cam, const int32_t* radius, const float* grad2d,
                                          float* dmean, float* dscale, float* dquat, float* dopacity,
                                          float* dfeat, gsr_stream_t stream) {
    (void)opacity;
    return backward_project_impl<false>(n, sh_degree, mean, scale, quat, feat, cam, radius, grad2d, dmean, dscale,
                                        dquat, dopacity, dfeat, stream);
}
