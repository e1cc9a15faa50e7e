// Status strings, loss, optimizer, and the L2 red microbenchmark.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "gsr_internal.cuh"

namespace gsr {

static thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e) {
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return GSR_ECUDA;
}

int check_launch() {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GSR_OK : cuda_fail(e);
}

namespace {

__global__ void l1_kernel(long long count, const float* __restrict__ img, const float* __restrict__ tgt,
                          float* __restrict__ grad, float* __restrict__ loss) {
    float acc = 0.0f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        float d = img[i] - tgt[i];
        grad[i] = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
        acc += fabsf(d);
    }
    if (!loss) return;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
    __shared__ float s[32];
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
        if (threadIdx.x == 0) atomicAdd(loss, acc);
    }
}

__global__ void adam_kernel(long long n, float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                            float eps, float bc1, float bc2) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.0f - b1) * gi;
        float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

__global__ void activate_kernel(long long n, const float* __restrict__ log_scale, const float* __restrict__ logit,
                                float* __restrict__ scale, float* __restrict__ opacity) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        scale[3 * i] = expf(log_scale[3 * i]);
        scale[3 * i + 1] = expf(log_scale[3 * i + 1]);
        scale[3 * i + 2] = expf(log_scale[3 * i + 2]);
        opacity[i] = 1.0f / (1.0f + expf(-logit[i]));
    }
}

__global__ void activate_backward_kernel(long long n, const float* __restrict__ scale,
                                         const float* __restrict__ opacity, const float* __restrict__ dscale,
                                         const float* __restrict__ dopacity, float* __restrict__ dlog_scale,
                                         float* __restrict__ dlogit) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        dlog_scale[3 * i] += dscale[3 * i] * scale[3 * i];
        dlog_scale[3 * i + 1] += dscale[3 * i + 1] * scale[3 * i + 1];
        dlog_scale[3 * i + 2] += dscale[3 * i + 2] * scale[3 * i + 2];
        const float o = opacity[i];
        dlogit[i] += dopacity[i] * o * (1.0f - o);
    }
}

// Access patterns of gsr_bench_red (see gsr.h): 0 own float per lane,
// 1 one float per warp, 2 nine lanes into one record per warp, 3 nine floats
// per lane into one record per warp, 4 own 16-byte slot per lane (v4),
// 5 two v4 and one scalar per lane into one record per warp, 6 nine floats
// per lane into the lane's own record.  Lanes >= `lanes` stay idle in the
// patterns with one address or record per warp (1, 3, 5).
__global__ void __launch_bounds__(256) red_bench_kernel(int pattern, int lanes, int iters, float* __restrict__ buf,
                                                        long long nfloats) {
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long gwarp = gtid >> 5;
    const int lane = threadIdx.x & 31;
    const long long nrec = nfloats / GSR_REC;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const long long nwarps = nthreads >> 5;
    const bool idle = (pattern == 1 || pattern == 3 || pattern == 5) && lane >= lanes;
    for (int it = 0; it < iters && !idle; ++it) {
        const long long w = (gwarp + (long long)it * nwarps) % nrec;  // record touched by this warp
        float* rec = buf + w * GSR_REC;
        const long long t = gtid + (long long)it * nthreads;          // this lane's running index
        if (pattern == 0) {
            red_add(buf + t % nfloats, 1.0f);
        } else if (pattern == 1) {
            red_add(rec, 1.0f);
        } else if (pattern == 2) {
            if (lane < 9) red_add(rec + lane, 1.0f);
        } else if (pattern == 3) {
#pragma unroll
            for (int q = 0; q < 9; ++q) red_add(rec + q, 1.0f);
        } else if (pattern == 4) {
            red_add_v4(buf + 4 * (t % (nfloats / 4)), 1.0f, 1.0f, 1.0f, 1.0f);
        } else if (pattern == 5) {
            red_add_v4(rec, 1.0f, 1.0f, 1.0f, 1.0f);
            red_add_v4(rec + 4, 1.0f, 1.0f, 1.0f, 1.0f);
            red_add(rec + 8, 1.0f);
        } else {
            float* own = buf + (t % nrec) * GSR_REC;
#pragma unroll
            for (int q = 0; q < 9; ++q) red_add(own + q, 1.0f);
        }
    }
}

}  // namespace
}  // namespace gsr

using namespace gsr;

extern "C" const char* gsr_status_string(int status) {
    switch (status) {
        case GSR_OK: return "ok";
        case GSR_EINVAL: return "invalid argument";
        case GSR_ECAPACITY: return "duplicated keys exceed key_capacity";
        case GSR_ECUDA: return "CUDA error";
        case GSR_ETIMEOUT: return "reserved status (no call waits on the device)";
        case GSR_ESCRATCH: return "scratch buffer too small";
        case GSR_ELIMIT: return "size exceeds the fixed limit of the allocation-free variant";
        default: return "unknown status";
    }
}

extern "C" const char* gsr_last_cuda_error(void) { return g_cuda_err; }

extern "C" int gsr_version(void) { return 100; }

extern "C" int gsr_l1_loss(int64_t count, const float* image, const float* target, float* dL_dimage,
                           float* loss_sum, gsr_stream_t stream) {
    if (count < 0 || (count > 0 && (!image || !target || !dL_dimage))) return GSR_EINVAL;
    if (count == 0) return GSR_OK;
    long long blocks = (count + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    l1_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(count, image, target, dL_dimage, loss_sum);
    return check_launch();
}

extern "C" int gsr_adam_step(int64_t n, float* param, const float* grad, float* m, float* v, float lr,
                             float beta1, float beta2, float eps, int32_t step, gsr_stream_t stream) {
    if (n < 0 || step < 1 || (n > 0 && (!param || !grad || !m || !v))) return GSR_EINVAL;
    if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f)) return GSR_EINVAL;
    if (n == 0) return GSR_OK;
    float bc1 = (float)(1.0 - pow((double)beta1, (double)step));
    float bc2 = (float)(1.0 - pow((double)beta2, (double)step));
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    adam_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(n, param, grad, m, v, lr, beta1, beta2, eps,
                                                                bc1, bc2);
    return check_launch();
}

extern "C" int gsr_bench_red(int32_t pattern, int32_t active_lanes, int32_t blocks, int32_t iters, float* buffer,
                             int64_t buffer_floats, int64_t* adds, gsr_stream_t stream) {
    if (pattern < 0 || pattern > 6 || blocks <= 0 || iters <= 0 || !buffer || buffer_floats < 32 * GSR_REC || !adds)
        return GSR_EINVAL;
    if (active_lanes < 1 || active_lanes > 32) return GSR_EINVAL;
    if (!aligned16(buffer)) return GSR_EINVAL;  // 16-byte records and slots (vector reds)
    const long long threads = (long long)blocks * 256, warps = threads / 32;
    const bool per_warp = pattern == 1 || pattern == 3 || pattern == 5;
    const long long lanes = per_warp ? warps * active_lanes : threads;  // lanes that send
    const long long per_lane[7] = {1, 1, 0, 9, 4, 9, 9};
    const long long per_iter = pattern == 2 ? warps * 9 : lanes * per_lane[pattern];
    *adds = per_iter * iters;
    red_bench_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(pattern, active_lanes, iters, buffer, buffer_floats);
    return check_launch();
}

extern "C" int gsr_activate(int64_t n, const float* log_scale, const float* opacity_logit, float* scale,
                            float* opacity, gsr_stream_t stream) {
    if (n < 0 || (n > 0 && (!log_scale || !opacity_logit || !scale || !opacity))) return GSR_EINVAL;
    if (n == 0) return GSR_OK;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    activate_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(n, log_scale, opacity_logit, scale, opacity);
    return check_launch();
}

extern "C" int gsr_activate_backward(int64_t n, const float* scale, const float* opacity, const float* dscale,
                                     const float* dopacity, float* dlog_scale, float* dopacity_logit,
                                     gsr_stream_t stream) {
    if (n < 0 || (n > 0 && (!scale || !opacity || !dscale || !dopacity || !dlog_scale || !dopacity_logit)))
        return GSR_EINVAL;
    if (n == 0) return GSR_OK;
    long long blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    activate_backward_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(n, scale, opacity, dscale, dopacity,
                                                                             dlog_scale, dopacity_logit);
    return check_launch();
}
