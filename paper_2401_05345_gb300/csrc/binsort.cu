// Tile binning through the CUDA Toolkit's CUB radix sort: the comparison arm
// of the hand-written binning (same outputs), and the allocation-free
// variant, whose scratch is a static device array.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <mutex>

#include "gsr_internal.cuh"

namespace gsr {
namespace {

struct BinGeom {
    int W, H, tw, th, gx, gy, twl, thl, tiles, end_bit;
};

int ilog2(int x) { int l = 0; while ((1 << l) < x) ++l; return l; }

bool make_geom(int W, int H, int tw, int th, BinGeom& g) {
    if (W <= 0 || H <= 0) return false;
    if (!pow2_in(tw, 8, 32) || !pow2_in(th, 8, 32) || tw * th > 512) return false;
    g.W = W; g.H = H; g.tw = tw; g.th = th;
    g.gx = (W + tw - 1) / tw;
    g.gy = (H + th - 1) / th;
    g.twl = ilog2(tw); g.thl = ilog2(th);
    g.tiles = g.gx * g.gy;
    int bits = 0;
    while ((1ll << bits) < (long long)g.tiles) ++bits;
    g.end_bit = 32 + (bits > 0 ? bits : 1);
    return true;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

__global__ void count_kernel(int n, const float* __restrict__ splat2d, const int* __restrict__ radius,
                             BinGeom g, uint32_t* __restrict__ counts) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > n) return;
    uint32_t c = 0;
    if (i < n) {
        int r = radius[i];
        if (r > 0) {
            float2 uv = *reinterpret_cast<const float2*>(splat2d + (size_t)i * GSR_REC);
            int x0, x1, y0, y1;
            tile_rect(uv.x, uv.y, r, g.gx, g.gy, g.twl, g.thl, x0, x1, y0, y1);
            int nt = (x1 - x0) * (y1 - y0);
            c = nt > 0 ? (uint32_t)nt : 0u;
        }
    }
    counts[i] = c;  // counts[n] = 0 so the exclusive scan ends with the total
}

__global__ void duplicate_kernel(int n, const float* __restrict__ splat2d, const int* __restrict__ radius,
                                 BinGeom g, const uint32_t* __restrict__ offsets,
                                 uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int r = radius[i];
    if (r <= 0) return;
    const float* rec = splat2d + (size_t)i * GSR_REC;
    int x0, x1, y0, y1;
    tile_rect(rec[0], rec[1], r, g.gx, g.gy, g.twl, g.thl, x0, x1, y0, y1);
    uint32_t o = offsets[i];
    uint64_t dbits = (uint64_t)__float_as_uint(rec[9]);
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) {
            keys[o] = ((uint64_t)(uint32_t)(y * g.gx + x) << 32) | dbits;
            vals[o] = (uint32_t)i;
            ++o;
        }
}

__global__ void ranges_kernel(long long nkeys, const uint64_t* __restrict__ keys, uint32_t* __restrict__ ranges) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkeys) return;
    uint32_t t = (uint32_t)(keys[k] >> 32);
    if (k == 0 || (uint32_t)(keys[k - 1] >> 32) != t) ranges[2 * (size_t)t] = (uint32_t)k;
    if (k == nkeys - 1 || (uint32_t)(keys[k + 1] >> 32) != t) ranges[2 * (size_t)t + 1] = (uint32_t)(k + 1);
}

// ---- two-stage binning: depth order first, then a short tile-id sort -----
// Sorting the Gaussians once by depth (stable, so equal depths keep id order)
// and emitting their tile entries in that order leaves only the tile id to
// sort: a stable radix sort over ceil(log2(tiles)) bits gives exactly the
// order of the (tile << 32 | depth) sort with id tie-break, in 2 passes over
// the duplicated entries instead of 6.
struct Scratch2 {
    uint32_t *dkeys_in, *dkeys_out, *ids_in, *order, *counts;
    uint32_t *tkeys_in, *tkeys_out, *vals_in;
    void* cub_tmp;
    size_t cub_bytes, total;
};

int layout2(int n, long long cap, int tile_bits, char* base, Scratch2& s) {
    size_t a = 0, b = 0, c = 0;
    const int nn = n > 0 ? n : 1;
    const int cc = (int)(cap > 0 ? cap : 1);
    cudaError_t e = cub::DeviceRadixSort::SortPairs(nullptr, a, (uint32_t*)nullptr, (uint32_t*)nullptr,
                                                    (uint32_t*)nullptr, (uint32_t*)nullptr, nn, 0, 32);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cub::DeviceScan::ExclusiveSum(nullptr, b, (uint32_t*)nullptr, (uint32_t*)nullptr, nn + 1);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cub::DeviceRadixSort::SortPairs(nullptr, c, (uint32_t*)nullptr, (uint32_t*)nullptr, (uint32_t*)nullptr,
                                        (uint32_t*)nullptr, cc, 0, tile_bits);
    if (e != cudaSuccess) return cuda_fail(e);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return base ? base + o : nullptr; };
    const size_t vn = sizeof(uint32_t) * (size_t)nn, vc = sizeof(uint32_t) * (size_t)cc;
    s.dkeys_in = (uint32_t*)take(vn);
    s.dkeys_out = (uint32_t*)take(vn);
    s.ids_in = (uint32_t*)take(vn);
    s.order = (uint32_t*)take(vn);
    s.counts = (uint32_t*)take(sizeof(uint32_t) * ((size_t)nn + 1));
    s.tkeys_in = (uint32_t*)take(vc);
    s.tkeys_out = (uint32_t*)take(vc);
    s.vals_in = (uint32_t*)take(vc);
    s.cub_bytes = a > b ? (a > c ? a : c) : (b > c ? b : c);
    s.cub_tmp = take(s.cub_bytes);
    s.total = off;
    return GSR_OK;
}

int tile_bits_of(const BinGeom& g) {
    int bits = 1;
    while ((1ll << bits) < (long long)g.tiles) ++bits;
    return bits;
}

__global__ void depth_keys_kernel(int n, const float* __restrict__ splat2d, const int* __restrict__ radius,
                                  uint32_t* __restrict__ keys, uint32_t* __restrict__ ids) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = radius[i] > 0 ? __float_as_uint(splat2d[(size_t)i * GSR_REC + 9]) : 0xffffffffu;
    ids[i] = (uint32_t)i;
}

__global__ void count_sorted_kernel(int n, const float* __restrict__ splat2d, const int* __restrict__ radius,
                                    const uint32_t* __restrict__ order, BinGeom g, uint32_t* __restrict__ counts) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > n) return;
    uint32_t c = 0;
    if (j < n) {
        const uint32_t i = order[j];
        const int r = radius[i];
        if (r > 0) {
            float2 uv = *reinterpret_cast<const float2*>(splat2d + (size_t)i * GSR_REC);
            int x0, x1, y0, y1;
            tile_rect(uv.x, uv.y, r, g.gx, g.gy, g.twl, g.thl, x0, x1, y0, y1);
            const int nt = (x1 - x0) * (y1 - y0);
            c = nt > 0 ? (uint32_t)nt : 0u;
        }
    }
    counts[j] = c;
}

// Writes every visible Gaussian's tile entries (depth rank j, tiles
// row-major inside its rectangle).  A warp takes 32 consecutive ranks, whose
// entries form one contiguous range, and its lanes write that range together
// (entry e goes to the lane whose prefix interval holds it), so the stores
// are coalesced whatever the per-Gaussian counts.
__global__ void __launch_bounds__(256)
duplicate_sorted_kernel(int n, const float* __restrict__ splat2d, const int* __restrict__ radius,
                        const uint32_t* __restrict__ order, BinGeom g, const uint32_t* __restrict__ offsets,
                        uint32_t* __restrict__ tkeys, uint32_t* __restrict__ vals) {
    __shared__ uint32_t s_pre[8][33];
    __shared__ int s_x0[8][32], s_wd[8][32], s_y0[8][32];
    __shared__ uint32_t s_id[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int j0 = j - lane;
    if (j0 >= n) return;  // whole warp past the end
    uint32_t c = 0, id = 0;
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    if (j < n) {
        id = order[j];
        const int r = radius[id];
        if (r > 0) {
            float2 uv = *reinterpret_cast<const float2*>(splat2d + (size_t)id * GSR_REC);
            tile_rect(uv.x, uv.y, r, g.gx, g.gy, g.twl, g.thl, x0, x1, y0, y1);
            const int nt = (x1 - x0) * (y1 - y0);
            c = nt > 0 ? (uint32_t)nt : 0u;
        }
    }
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    s_pre[w][lane] = incl - c;
    if (lane == 31) s_pre[w][32] = incl;
    s_x0[w][lane] = x0;
    s_wd[w][lane] = x1 - x0;
    s_y0[w][lane] = y0;
    s_id[w][lane] = id;
    __syncwarp();
    const uint32_t total = s_pre[w][32];
    const uint32_t base = offsets[j0];
    for (uint32_t e = lane; e < total; e += 32) {
        int lo = 0, hi = 31;  // last lane whose prefix start <= e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_pre[w][mid] <= e) lo = mid; else hi = mid - 1;
        }
        const uint32_t local = e - s_pre[w][lo];
        const int wd = s_wd[w][lo];
        const int ty = s_y0[w][lo] + (int)(local / (uint32_t)wd);
        const int tx = s_x0[w][lo] + (int)(local % (uint32_t)wd);
        tkeys[base + e] = (uint32_t)(ty * g.gx + tx);
        vals[base + e] = s_id[w][lo];
    }
}

__global__ void ranges_tile_kernel(long long nkeys, const uint32_t* __restrict__ tkeys, uint32_t* __restrict__ ranges) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkeys) return;
    const uint32_t t = tkeys[k];
    if (k == 0 || tkeys[k - 1] != t) ranges[2 * (size_t)t] = (uint32_t)k;
    if (k == nkeys - 1 || tkeys[k + 1] != t) ranges[2 * (size_t)t + 1] = (uint32_t)(k + 1);
}

__global__ void full_keys_kernel(long long nkeys, const uint32_t* __restrict__ tkeys,
                                 const uint32_t* __restrict__ point_list, const float* __restrict__ splat2d,
                                 uint64_t* __restrict__ keys) {
    long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkeys) return;
    keys[k] = ((uint64_t)tkeys[k] << 32) | (uint64_t)__float_as_uint(splat2d[(size_t)point_list[k] * GSR_REC + 9]);
}

}  // namespace
}  // namespace gsr

using namespace gsr;

extern "C" int gsr_bin_scratch_bytes_library(int32_t n, int32_t width, int32_t height, int32_t tile_w,
                                     int32_t tile_h, int64_t key_capacity, size_t* bytes) {
    BinGeom g;
    if (n < 0 || key_capacity < 0 || key_capacity >= 0xffffffffll || !bytes ||
        !make_geom(width, height, tile_w, tile_h, g))
        return GSR_EINVAL;
    Scratch2 s;
    int rc = layout2(n, key_capacity, tile_bits_of(g), nullptr, s);
    if (rc != GSR_OK) return rc;
    *bytes = s.total;
    return GSR_OK;
}

extern "C" int gsr_bin_sort_library(int32_t n, int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                            const float* splat2d, const int32_t* radius, int64_t key_capacity,
                            void* scratch, size_t scratch_bytes, uint32_t* point_list,
                            uint32_t* tile_ranges, uint64_t* keys_out, int64_t* n_keys,
                            gsr_stream_t stream_) {
    BinGeom g;
    if (n < 0 || key_capacity < 0 || key_capacity >= 0xffffffffll || !n_keys ||
        !make_geom(width, height, tile_w, tile_h, g))
        return GSR_EINVAL;
    if (!tile_ranges || !scratch || (n > 0 && (!splat2d || !radius)) || (key_capacity > 0 && !point_list))
        return GSR_EINVAL;
    if (!aligned16(splat2d) || !aligned16(scratch) || (keys_out && !aligned8(keys_out))) return GSR_EINVAL;
    cudaStream_t stream = (cudaStream_t)stream_;
    const int tbits = tile_bits_of(g);
    Scratch2 s;
    int rc = layout2(n, key_capacity, tbits, (char*)scratch, s);
    if (rc != GSR_OK) return rc;
    if (scratch_bytes < s.total) return GSR_ESCRATCH;
    cudaError_t e = cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)g.tiles, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    *n_keys = 0;
    if (n == 0) return GSR_OK;
    // 1. Gaussians in (depth, id) order
    depth_keys_kernel<<<(n + 255) / 256, 256, 0, stream>>>(n, splat2d, radius, s.dkeys_in, s.ids_in);
    if ((rc = check_launch()) != GSR_OK) return rc;
    size_t tb = s.cub_bytes;
    e = cub::DeviceRadixSort::SortPairs(s.cub_tmp, tb, s.dkeys_in, s.dkeys_out, s.ids_in, s.order, n, 0, 32, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    // 2. tiles touched, in that order, and their offsets
    count_sorted_kernel<<<(n + 1 + 255) / 256, 256, 0, stream>>>(n, splat2d, radius, s.order, g, s.counts);
    if ((rc = check_launch()) != GSR_OK) return rc;
    tb = s.cub_bytes;
    e = cub::DeviceScan::ExclusiveSum(s.cub_tmp, tb, s.counts, s.counts, n + 1, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    uint32_t total = 0;
    e = cudaMemcpyAsync(&total, s.counts + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e);
    *n_keys = (int64_t)total;
    if ((long long)total > key_capacity) return GSR_ECAPACITY;
    if (total == 0) return GSR_OK;
    // 3. entries emitted in depth order, then a stable sort on the tile id
    duplicate_sorted_kernel<<<(n + 255) / 256, 256, 0, stream>>>(n, splat2d, radius, s.order, g, s.counts,
                                                                 s.tkeys_in, s.vals_in);
    if ((rc = check_launch()) != GSR_OK) return rc;
    tb = 0;
    e = cub::DeviceRadixSort::SortPairs(nullptr, tb, s.tkeys_in, s.tkeys_out, s.vals_in, point_list, (int)total, 0,
                                        tbits, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    if (tb > s.cub_bytes) return GSR_ESCRATCH;
    tb = s.cub_bytes;
    e = cub::DeviceRadixSort::SortPairs(s.cub_tmp, tb, s.tkeys_in, s.tkeys_out, s.vals_in, point_list, (int)total,
                                        0, tbits, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    const unsigned blocks = (unsigned)((total + 255) / 256);
    ranges_tile_kernel<<<blocks, 256, 0, stream>>>((long long)total, s.tkeys_out, tile_ranges);
    if ((rc = check_launch()) != GSR_OK) return rc;
    if (keys_out) {
        full_keys_kernel<<<blocks, 256, 0, stream>>>((long long)total, s.tkeys_out, point_list, splat2d, keys_out);
        if ((rc = check_launch()) != GSR_OK) return rc;
    }
    return GSR_OK;
}

extern "C" int gsr_entry_offsets_scratch_bytes(int32_t n, size_t* bytes) {
    if (n < 0 || !bytes) return GSR_EINVAL;
    size_t b = 0;
    cudaError_t e = cub::DeviceScan::ExclusiveSum(nullptr, b, (uint32_t*)nullptr, (uint32_t*)nullptr, n + 1);
    if (e != cudaSuccess) return cuda_fail(e);
    *bytes = b > 0 ? b : 1;
    return GSR_OK;
}

extern "C" int gsr_entry_offsets(int32_t n, int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                                 const float* splat2d, const int32_t* radius, void* scratch, size_t scratch_bytes,
                                 uint32_t* offsets, gsr_stream_t stream_) {
    BinGeom g;
    if (n < 0 || !offsets || !scratch || !make_geom(width, height, tile_w, tile_h, g)) return GSR_EINVAL;
    if (n > 0 && (!splat2d || !radius || !aligned16(splat2d))) return GSR_EINVAL;
    size_t need = 0;
    int rc = gsr_entry_offsets_scratch_bytes(n, &need);
    if (rc != GSR_OK) return rc;
    if (scratch_bytes < need) return GSR_ESCRATCH;
    cudaStream_t s = (cudaStream_t)stream_;
    count_kernel<<<(n + 1 + 255) / 256, 256, 0, s>>>(n, splat2d, radius, g, offsets);
    if ((rc = check_launch()) != GSR_OK) return rc;
    size_t tb = scratch_bytes;
    cudaError_t e = cub::DeviceScan::ExclusiveSum(scratch, tb, offsets, offsets, n + 1, s);
    return e == cudaSuccess ? GSR_OK : cuda_fail(e);
}

// ----------------------------------------------------------------------------
// Allocation-free variant of gsr_bin_sort.
//
// Some callers cannot allocate device memory at all: code that runs where the
// host process has handed every byte of the GPU to another allocator (a
// framework's caching pool, an embedding application with a fixed budget),
// or real-time loops that must never pay cudaMalloc's latency and implicit
// device synchronisation.  For them the scratch of the binning lives in one
// static device array inside this library, reserved when the library's
// device code is loaded on a GPU and held until the process exits.
// ----------------------------------------------------------------------------
namespace gsr {
namespace {

constexpr size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kStaticCountsBytes = round256(sizeof(uint32_t) * ((size_t)GSR_STATIC_BIN_MAX_GAUSSIANS + 1));
constexpr size_t kStaticKeysBytes = sizeof(uint64_t) * (size_t)GSR_STATIC_BIN_MAX_KEYS;
constexpr size_t kStaticValsBytes = sizeof(uint32_t) * (size_t)GSR_STATIC_BIN_MAX_KEYS;
constexpr size_t kStaticCubBytes = (size_t)8 << 20;
constexpr size_t kStaticBytes = kStaticCountsBytes + kStaticKeysBytes + kStaticValsBytes + kStaticCubBytes;

// Shared by every call on a device; contents persist between calls.
static __device__ __align__(256) unsigned char g_bin_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
unsigned char* g_static_ptr[kMaxDevices] = {};

// Device address of g_bin_scratch on the current device (looked up once per
// device; the host-side symbol is only a stand-in for it).
int static_scratch(unsigned char** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= kMaxDevices) return GSR_EINVAL;
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess) return cuda_fail(e);
        // CUB's own temporary storage for the largest problem must fit its slice
        size_t scan_b = 0, sort_b = 0;
        cub::DoubleBuffer<uint64_t> kb(nullptr, nullptr);
        cub::DoubleBuffer<uint32_t> vb(nullptr, nullptr);
        e = cub::DeviceScan::ExclusiveSum(nullptr, scan_b, (uint32_t*)nullptr, (uint32_t*)nullptr,
                                          GSR_STATIC_BIN_MAX_GAUSSIANS + 1);
        if (e != cudaSuccess) return cuda_fail(e);
        e = cub::DeviceRadixSort::SortPairs(nullptr, sort_b, kb, vb, GSR_STATIC_BIN_MAX_KEYS, 0, 64);
        if (e != cudaSuccess) return cuda_fail(e);
        if (scan_b > kStaticCubBytes || sort_b > kStaticCubBytes) return GSR_ESCRATCH;
        g_static_ptr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_static_ptr[dev];
    return GSR_OK;
}

}  // namespace
}  // namespace gsr

extern "C" int gsr_bin_sort_static(int32_t n, int32_t width, int32_t height, int32_t tile_w,
                                   int32_t tile_h, const float* splat2d, const int32_t* radius,
                                   int64_t key_capacity, uint32_t* point_list, uint32_t* tile_ranges,
                                   uint64_t* keys_out, int64_t* n_keys, gsr_stream_t stream_) {
    BinGeom g;
    if (n < 0 || key_capacity < 0 || key_capacity >= 0xffffffffll || !n_keys ||
        !make_geom(width, height, tile_w, tile_h, g))
        return GSR_EINVAL;
    if (n > GSR_STATIC_BIN_MAX_GAUSSIANS) return GSR_ELIMIT;
    if (!tile_ranges || (n > 0 && (!splat2d || !radius)) || (key_capacity > 0 && (!point_list || !keys_out)))
        return GSR_EINVAL;
    if (!aligned16(splat2d) || (keys_out && !aligned8(keys_out))) return GSR_EINVAL;
    unsigned char* base = nullptr;
    int rc = static_scratch(&base);
    if (rc != GSR_OK) return rc;
    uint32_t* counts = reinterpret_cast<uint32_t*>(base);
    uint64_t* keys_tmp = reinterpret_cast<uint64_t*>(base + kStaticCountsBytes);
    uint32_t* vals_tmp = reinterpret_cast<uint32_t*>(base + kStaticCountsBytes + kStaticKeysBytes);
    void* cub_tmp = base + kStaticCountsBytes + kStaticKeysBytes + kStaticValsBytes;

    cudaStream_t stream = (cudaStream_t)stream_;
    cudaError_t e = cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)g.tiles, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    *n_keys = 0;
    if (n == 0) return GSR_OK;
    // every counts[0..n] is written here, so nothing left by an earlier call is read
    count_kernel<<<(n + 1 + 255) / 256, 256, 0, stream>>>(n, splat2d, radius, g, counts);
    if ((rc = check_launch()) != GSR_OK) return rc;
    size_t tb = kStaticCubBytes;
    e = cub::DeviceScan::ExclusiveSum(cub_tmp, tb, counts, counts, n + 1, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    uint32_t total = 0;
    e = cudaMemcpyAsync(&total, counts + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e);
    *n_keys = (int64_t)total;
    if ((long long)total > key_capacity) return GSR_ECAPACITY;
    if ((long long)total > GSR_STATIC_BIN_MAX_KEYS) return GSR_ELIMIT;
    if (total == 0) return GSR_OK;
    duplicate_kernel<<<(n + 255) / 256, 256, 0, stream>>>(n, splat2d, radius, g, counts, keys_tmp, vals_tmp);
    if ((rc = check_launch()) != GSR_OK) return rc;
    // double-buffered sort: the caller's outputs serve as the alternate buffers
    cub::DoubleBuffer<uint64_t> kb(keys_tmp, keys_out);
    cub::DoubleBuffer<uint32_t> vb(vals_tmp, point_list);
    tb = kStaticCubBytes;
    e = cub::DeviceRadixSort::SortPairs(cub_tmp, tb, kb, vb, (int)total, 0, g.end_bit, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    if (kb.Current() != keys_out) {
        e = cudaMemcpyAsync(keys_out, kb.Current(), sizeof(uint64_t) * total, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (vb.Current() != point_list) {
        e = cudaMemcpyAsync(point_list, vb.Current(), sizeof(uint32_t) * total, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    ranges_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>((long long)total, keys_out, tile_ranges);
    return check_launch();
}
