// Batched backward over many views: longest-first work order and one
// persistent launch (kernels in raster_common.cuh).
#include <cub/device/device_radix_sort.cuh>

#include "raster_common.cuh"

namespace gsr {
int check_bwd_opts(const gsr_backward_opts& o);

namespace {

// Persistent backward over many views: each CTA takes (view, tile) items in
// the given order (longest tile lists first) from one atomic counter until
// the list is exhausted.  No CTA waits on another.
template <class SH, int MODE, bool STORE_T>
__global__ void __launch_bounds__(SH::NT)
backward_batched_kernel(const gsr_view* __restrict__ views, const uint32_t* __restrict__ items, int n_items,
                        unsigned* __restrict__ counter, int threshold) {
    __shared__ BwdSmem<SH::B, MODE> sm;
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
        p.g = RasterGeom{v.width, v.height, (v.width + 15) / 16, (v.height + 15) / 16};
        p.ranges = reinterpret_cast<const uint2*>(v.tile_ranges);
        p.point_list = v.point_list;
        p.splat2d = v.splat2d;
        p.bg0 = v.bg[0]; p.bg1 = v.bg[1]; p.bg2 = v.bg[2];
        p.final_T = v.final_T;
        p.n_contrib = v.n_contrib;
        p.dL_dimage = v.dL_dimage;
        p.grad2d = v.grad2d;
        p.threshold = threshold;
        p.order = nullptr;  // the item list is the order
        p.block_mask = v.block_mask;
        backward_tile<SH, MODE, STORE_T>(p, (int)(code & 0xffffffu), sm);
    }
}

// Sort keys of the batched work order: larger tile lists first.
__global__ void batch_keys_kernel(int n_views, const gsr_view* __restrict__ views, const int* __restrict__ offsets,
                                  int n_items, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
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

template <class SH, int MODE, bool STORE_T>
int launch_batched(int n_items, const gsr_view* views, const uint32_t* items, unsigned* counter, int thr,
                   int ctas_per_sm, cudaStream_t s) {
    auto k = backward_batched_kernel<SH, MODE, STORE_T>;
    int dev = 0, sms = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, SH::NT, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    const int per_sm = ctas_per_sm > 0 ? min(ctas_per_sm, max(occ, 1)) : max(occ, 1);
    k<<<sms * per_sm, SH::NT, 0, s>>>(views, items, n_items, counter, thr);
    return check_launch();
}

template <int MODE, int PPT>
int launch_batched_lay(int layout, bool store, int n_items, const gsr_view* views, const uint32_t* items,
                       unsigned* counter, int thr, int cps, cudaStream_t s) {
    if (layout == 0)
        return store ? launch_batched<Shape<16, 16, 0, PPT>, MODE, true>(n_items, views, items, counter, thr, cps, s)
                     : launch_batched<Shape<16, 16, 0, PPT>, MODE, false>(n_items, views, items, counter, thr, cps, s);
    return store ? launch_batched<Shape<16, 16, 1, PPT>, MODE, true>(n_items, views, items, counter, thr, cps, s)
                 : launch_batched<Shape<16, 16, 1, PPT>, MODE, false>(n_items, views, items, counter, thr, cps, s);
}

template <int MODE>
int launch_batched_mode(int ppt, int layout, bool store, int n_items, const gsr_view* views, const uint32_t* items,
                        unsigned* counter, int thr, int cps, cudaStream_t s) {
    if (ppt == 2) return launch_batched_lay<MODE, 2>(layout, store, n_items, views, items, counter, thr, cps, s);
    return launch_batched_lay<MODE, 1>(layout, store, n_items, views, items, counter, thr, cps, s);
}

size_t order_layout(int n_items, char* base, uint32_t** keys_in, uint32_t** keys_out, uint32_t** vals_in, void** tmp,
                    size_t* tmp_bytes) {
    size_t sort_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, (uint32_t*)nullptr, (uint32_t*)nullptr, (uint32_t*)nullptr,
                                    (uint32_t*)nullptr, n_items > 0 ? n_items : 1, 0, 32);
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

using namespace gsr;

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
    gsr_backward_opts o = {GSR_REDUCE_WARP, 0, 0, 1, 1, {0, 0, 0}};
    if (opts) o = *opts;
    if (n_views <= 0 || n_views > 256 || n_items < 0 || !views || !counter || (n_items > 0 && !items)) return GSR_EINVAL;
    if (check_bwd_opts(o) != GSR_OK || ctas_per_sm < 0) return GSR_EINVAL;
    if (o.reduce_mode == GSR_REDUCE_CLUSTER) return GSR_EINVAL;  // single-view launches only
    cudaStream_t s = (cudaStream_t)stream_;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (n_items == 0) return GSR_OK;
    const bool st = o.store_T != 0;
    const int ppt = o.pixels_per_thread == 2 ? 2 : 1;
    unsigned* c = (unsigned*)counter;
    switch (o.reduce_mode) {
        case GSR_REDUCE_PLAIN:
            return launch_batched_lay<GSR_REDUCE_PLAIN, 1>(o.lane_layout, st, n_items, views, items, c, o.threshold,
                                                           ctas_per_sm, s);
        case GSR_REDUCE_WARP:
            return launch_batched_mode<GSR_REDUCE_WARP>(ppt, o.lane_layout, st, n_items, views, items, c, o.threshold,
                                                        ctas_per_sm, s);
        case GSR_REDUCE_HYBRID:
            return launch_batched_mode<GSR_REDUCE_HYBRID>(ppt, o.lane_layout, st, n_items, views, items, c,
                                                          o.threshold, ctas_per_sm, s);
        default:
            return launch_batched_mode<GSR_REDUCE_BLOCK>(ppt, o.lane_layout, st, n_items, views, items, c,
                                                         o.threshold, ctas_per_sm, s);
    }
}
