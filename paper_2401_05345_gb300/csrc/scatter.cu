// Scatter-add of 9-value records with divergent destinations: the general
// form of the gradient accumulation, where the lanes of a warp may update
// different primitives (Sec. V-A1, the serialized reduction SW-S, used when
// warps cannot be made to update a single primitive, e.g. Pulsar's spheres).
#include "gsr_internal.cuh"

namespace gsr {
namespace {

__device__ __forceinline__ void load9(const float* __restrict__ v, float* x) {
#pragma unroll
    for (int q = 0; q < 9; ++q) x[q] = v[q];
}

// PLAIN: one atomic add per parameter per item.
// SERIAL: the lanes of a warp that share a destination form a group (a
//   match mask); a group of at least `threshold` lanes is reduced at the SM
//   (Sec. V-A1: one sum per destination instead of one atomic per lane),
//   smaller groups send each lane's reds to L2.  A reduced group shares its 9
//   parameters among its own lanes: every lane stages its values in shared
//   memory, and the lane of rank r in a group of g sums parameters r, r + g,
//   ... over the group's members (in lane order) and sends their reds.
//   Unreduced lanes send a record as two vector reds and one scalar red when
//   rows are 16-byte aligned, else as 9 scalar reds.
// SORTED: the warp's (destination, lane) pairs are sorted with a bitonic
//   network in registers, each lane fetches the values of its sorted
//   position, and a 5-step segmented shuffle scan leaves every group's total
//   with the group's last lane, which issues the 9 reds.
// The 9 reds of one record: with VEC (rows 16-byte aligned) two vector reds
// and one scalar red.
template <bool VEC>
__device__ __forceinline__ void red9(float* rec, const float* x) {
    if (VEC) {
        red_add_v4(rec, x[0], x[1], x[2], x[3]);
        red_add_v4(rec + 4, x[4], x[5], x[6], x[7]);
        red_add(rec + 8, x[8]);
    } else {
#pragma unroll
        for (int q = 0; q < 9; ++q) red_add(rec + q, x[q]);
    }
}

template <int METHOD, bool VEC>
__global__ void __launch_bounds__(256)
scatter9_kernel(long long n, const uint32_t* __restrict__ idx, const float* __restrict__ vals,
                float* __restrict__ out, int stride, int threshold) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const bool valid = i < n;
    const uint32_t d = valid ? idx[i] : 0xffffffffu;
    float x[9];
    if (valid) load9(vals + 9 * i, x);
    else
#pragma unroll
        for (int q = 0; q < 9; ++q) x[q] = 0.f;
    if (METHOD == 0) {
        if (valid) {
            float* rec = out + (size_t)d * stride;
#pragma unroll
            for (int q = 0; q < 9; ++q) atomicAdd(rec + q, x[q]);
        }
        return;
    }
    if constexpr (METHOD == 1) {
        __shared__ float s_x[8][32 * 9];  // per warp: lane-major values (stride 9: no bank conflicts)
        float* wx = s_x[threadIdx.x >> 5];
        const unsigned act = __ballot_sync(kFull, valid);
        const unsigned same = __match_any_sync(kFull, d) & act;
        const int g = __popc(same);
        const bool reduced = valid && g >= threshold;
        const unsigned red_lanes = __ballot_sync(kFull, reduced);
        if (!valid) return;
        float* rec = out + (size_t)d * stride;
        if (!reduced) {
            red9<VEC>(rec, x);
            return;
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) wx[lane * 9 + q] = x[q];
        __syncwarp(red_lanes);
        const int rank = __popc(same & ((1u << lane) - 1u));
        for (int q = rank; q < 9; q += g) {
            float sum = 0.0f;
            for (unsigned m = same; m; m &= m - 1u) sum += wx[(__ffs(m) - 1) * 9 + q];
            red_add(rec + q, sum);
        }
        return;
    }
    // METHOD 2: bitonic sort of (destination, source lane) over the warp
    uint32_t key = d, src = (uint32_t)lane;
    warp_sort_pairs(key, src, lane);
    float y[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) y[q] = __shfl_sync(kFull, x[q], (int)src);
    // segmented inclusive scan over runs of equal keys
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t kp = __shfl_up_sync(kFull, key, o);
        const bool same_run = lane >= o && kp == key;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float t = __shfl_up_sync(kFull, y[q], o);
            if (same_run) y[q] += t;
        }
    }
    const uint32_t kn = __shfl_down_sync(kFull, key, 1);
    const bool run_end = (lane == 31) || (kn != key);
    if (run_end && key != 0xffffffffu) red9<VEC>(out + (size_t)key * stride, y);
}

}  // namespace
}  // namespace gsr

using namespace gsr;

extern "C" int gsr_scatter_add9(int64_t n, const uint32_t* idx, const float* vals, float* out, int32_t stride,
                                int32_t method, int32_t threshold, gsr_stream_t stream) {
    if (n < 0 || (n > 0 && (!idx || !vals || !out)) || stride < 9 || method < 0 || method > 2 || threshold < 0 ||
        threshold > 33)
        return GSR_EINVAL;
    if (n == 0) return GSR_OK;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    cudaStream_t s = (cudaStream_t)stream;
    // the reduced methods send a record as vector reds when every row is 16-byte aligned
    const bool vec = (stride % 4) == 0 && aligned16(out);
    if (method == 0) scatter9_kernel<0, false><<<blocks, 256, 0, s>>>(n, idx, vals, out, stride, threshold);
    else if (method == 1 && vec) scatter9_kernel<1, true><<<blocks, 256, 0, s>>>(n, idx, vals, out, stride, threshold);
    else if (method == 1) scatter9_kernel<1, false><<<blocks, 256, 0, s>>>(n, idx, vals, out, stride, threshold);
    else if (vec) scatter9_kernel<2, true><<<blocks, 256, 0, s>>>(n, idx, vals, out, stride, threshold);
    else scatter9_kernel<2, false><<<blocks, 256, 0, s>>>(n, idx, vals, out, stride, threshold);
    return check_launch();
}
