// Tile binning with hand-written sorts: the per-tile, depth-ordered lists of
// splats that every pixel of a tile walks (Sec. III-A; the lists are the
// 3DGS rasterizer's, Sec. II-C).
//
// 1. Depth order.  The Gaussians are put in (depth, id) order by a stable LSD
//    radix sort of their 32-bit depth keys: three passes of 11, 11 and 10
//    bits.  Each pass is reduce-then-scan: per-tile digit counts (for the
//    first pass from the key-generation kernel, for the later ones added by
//    the previous pass's scatter as it writes each key), a column scan of
//    the [tile][digit] count matrix, and a scatter that ranks the tile's keys
//    with per-bit warp ballots.  No block waits on another.
// 2. Tile lists.  Walking the Gaussians in that order and appending each one
//    to the lists of the tiles its rectangle covers gives every tile's list
//    already in (depth, id) order, so the entries never go through a sort
//    of their own: a counting sort over tile ids places them directly.  The
//    entries, in depth order (tiles row-major inside a rectangle), are cut
//    into equal slices, one per warp of the placement grid (a Gaussian may
//    straddle two slices: it has one entry per tile, so order per tile is
//    kept).  One kernel counts each block's entries per tile (its
//    rectangles summed in a 2D difference array, then prefix-summed), a
//    column scan over the blocks gives every (block, tile) pair its first
//    slot (and the tile ranges), and a second pass writes the entries, one
//    rectangle row per lane and 32 rows per round per warp; rows of one tile
//    row that overlap take turns in lane (depth) order.
#include "gsr_internal.cuh"

namespace gsr {
namespace {

struct Geom {
    int W, H, tw, th, gx, gy, twl, thl, tiles;
};

int log2_exact(int x) { int l = 0; while ((1 << l) < x) ++l; return l; }

bool make_geom(int W, int H, int tw, int th, Geom& g) {
    if (W <= 0 || H <= 0) return false;
    if (!pow2_in(tw, 8, 32) || !pow2_in(th, 8, 32) || tw * th > 512) return false;
    g.W = W; g.H = H; g.tw = tw; g.th = th;
    g.gx = (W + tw - 1) / tw;
    g.gy = (H + th - 1) / th;
    if (g.gx >= 65536 || g.gy >= 65536) return false;  // tile coordinates are packed in 16 bits
    if ((long long)g.gx * g.gy >= (1ll << 31)) return false;
    g.twl = log2_exact(tw); g.thl = log2_exact(th);
    g.tiles = g.gx * g.gy;
    return true;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---- depth radix sort -------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 8;
constexpr int kRsTile = kRsThreads * kRsItems;  // keys per tile (block)
constexpr int kRsB0 = 11, kRsB1 = 11, kRsB2 = 10;
constexpr int kRsS1 = kRsB0, kRsS2 = kRsB0 + kRsB1;

int rs_tiles(int n) { return (n + kRsTile - 1) / kRsTile; }

// Exclusive scan of one value per thread over a 256-thread block (returns
// the thread's prefix; *total receives the block sum).  s_wsum: 8 words.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_wsum, uint32_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_wsum[w] = incl;
    __syncthreads();
    uint32_t woff = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < kRsWarps; ++q) {
        const uint32_t x = s_wsum[q];
        woff += q < w ? x : 0u;
        tot += x;
    }
    __syncthreads();  // s_wsum may be reused by the caller
    *total = tot;
    return woff + incl - v;
}

// The lanes of `active` whose label has the same low BITS bits as this
// lane's: one ballot per bit, each keeping the lanes that agree on it.
template <int BITS>
__device__ __forceinline__ unsigned match_low_bits(uint32_t label, unsigned active) {
    unsigned m = active;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const bool bit = (label >> b) & 1u;
        const unsigned v = __ballot_sync(kFull, bit);
        m &= bit ? v : ~v;
    }
    return m;
}

// Depth keys (FP32 bits of the camera depth, positive, so their unsigned
// order is the numeric order) and ids; per-tile counts of the first digit.
// A culled Gaussian gets the key 2^31 + its id: above every finite depth (so
// culled Gaussians sort after all others, in any order, and bin nowhere) and
// distinct, so their digits spread over the count matrices instead of all
// adding to one counter per pass.
__global__ void __launch_bounds__(kRsThreads)
depth_keys_kernel(int n, const float* __restrict__ splat2d, const int* __restrict__ radius,
                  uint32_t* __restrict__ keys, uint32_t* __restrict__ ids, uint32_t* __restrict__ counts0) {
    constexpr int NB = 1 << kRsB0;
    __shared__ uint32_t h[NB];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long first = (long long)blockIdx.x * kRsTile + w * 32 * kRsItems + lane;
    int rad[kRsItems];
    float dep[kRsItems];
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {  // every load issued before the first use
        const long long i = first + 32 * it;
        rad[it] = i < n ? radius[i] : 0;
        dep[it] = i < n ? splat2d[(size_t)i * GSR_REC + 9] : 0.0f;
    }
    for (int i = threadIdx.x; i < NB; i += kRsThreads) h[i] = 0;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        const long long i = first + 32 * it;
        if (i < n) {
            const uint32_t k = rad[it] > 0 ? __float_as_uint(dep[it]) : (0x80000000u | (uint32_t)i);
            keys[i] = k;
            ids[i] = (uint32_t)i;
            atomicAdd(&h[k & (NB - 1)], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NB; i += kRsThreads) counts0[(size_t)blockIdx.x * NB + i] = h[i];
}

// In-place exclusive scan down the columns of a [rows][cols] matrix, with
// the column totals.  Block: 32 columns x 32 row segments.  When ranges is
// given, the last block to finish also scans the totals over the columns
// (tile start offsets), writes the [start, end) ranges (0,0 for empty
// columns) and the grand total (info[0], and count_out[0] with a status in
// count_out[1]: 0 ok, 1 more than cap, 2 inconsistent counts; all ranges
// empty unless 0).
__global__ void __launch_bounds__(1024)
colscan_kernel(int rows, int cols, uint32_t* __restrict__ m, uint32_t* __restrict__ tot,
               uint32_t* __restrict__ start, uint32_t* __restrict__ ranges, uint32_t* __restrict__ info,
               uint32_t cap, uint32_t* __restrict__ count_out, uint32_t* __restrict__ order) {
    __shared__ uint32_t s_seg[32][33];
    __shared__ bool s_last;
    const int cx = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + cx;
    const int per = (rows + 31) / 32;
    const int r0 = seg * per, r1 = min(rows, r0 + per);
    constexpr int kHeld = 16;  // segments up to this long are read once and kept in registers
    const bool held = per <= kHeld;
    uint32_t v[kHeld];
    uint32_t sum = 0;
    if (c < cols) {
        if (held) {
#pragma unroll
            for (int q = 0; q < kHeld; ++q) {
                v[q] = r0 + q < r1 ? m[(size_t)(r0 + q) * cols + c] : 0u;
                sum += v[q];
            }
        } else {
#pragma unroll 4
            for (int r = r0; r < r1; ++r) sum += m[(size_t)r * cols + c];
        }
    }
    s_seg[seg][cx] = sum;
    __syncthreads();
    {   // exclusive scan over the segments: warp `seg` takes column `seg`, lane `cx` its segment `cx`
        const uint32_t x = s_seg[cx][seg];
        uint32_t incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (cx >= o) incl += t;
        }
        s_seg[cx][seg] = incl - x;
        const int cc = blockIdx.x * 32 + seg;
        if (cx == 31 && cc < cols) {
            tot[cc] = incl;
            if (ranges) __threadfence();  // the totals are what the last block reads
        }
    }
    __syncthreads();
    if (c < cols) {
        uint32_t run = s_seg[seg][cx];
        if (held) {
#pragma unroll
            for (int q = 0; q < kHeld; ++q) {
                if (r0 + q < r1) m[(size_t)(r0 + q) * cols + c] = run;
                run += v[q];
            }
        } else {
#pragma unroll 4
            for (int r = r0; r < r1; ++r) {
                const size_t o = (size_t)r * cols + c;
                const uint32_t x = m[o];
                m[o] = run;
                run += x;
            }
        }
    }
    if (!ranges) return;
    // last block: exclusive scan of the column totals
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&info[2], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    uint32_t carry = 0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < cols; base += 1024 * 4) {
        const int c0 = base + threadIdx.x * 4;
        uint32_t v[4], s = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = c0 + j < cols ? __ldcg(tot + c0 + j) : 0u;
            s += v[j];
        }
        uint32_t incl = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_seg[0][w] = incl;
        __syncthreads();
        // the 32 warp sums, scanned across one warp's lanes by every warp
        const uint32_t ws = s_seg[0][lane];
        uint32_t wincl = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, wincl, o);
            if (lane >= o) wincl += t;
        }
        const uint32_t woff = __shfl_sync(kFull, wincl - ws, w), btot = __shfl_sync(kFull, wincl, 31);
        __syncthreads();
        uint32_t run = carry + woff + incl - s;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (c0 + j < cols) {
                start[c0 + j] = run;
                ranges[2 * (size_t)(c0 + j)] = v[j] ? run : 0u;
                ranges[2 * (size_t)(c0 + j) + 1] = v[j] ? run + v[j] : 0u;
            }
            run += v[j];
        }
        carry += btot;
    }
    // more keys than the caller's capacity (or inconsistent counts): every
    // range empty, so nothing downstream reads the lists
    const uint32_t status = (info[1] || carry != __ldcg(info + 4)) ? 2u : (carry > cap ? 1u : 0u);
    if (status)
        for (int c = threadIdx.x; c < cols; c += 1024) {
            ranges[2 * (size_t)c] = 0u;
            ranges[2 * (size_t)c + 1] = 0u;
        }
    if (threadIdx.x == 0) {
        info[0] = carry;
        if (count_out) {
            count_out[0] = carry;
            count_out[1] = status;
        }
    }
    if (order) {  // the longest-first tile order of the ranges just written
        __syncthreads();
        tile_order_block(cols, reinterpret_cast<const uint2*>(ranges), order, &s_seg[0][0]);
    }
}

// One scatter pass of the depth sort.  The tile's keys are ranked stably
// (warp-striped: warp w holds keys w*256 .. w*256+255 of the tile, item i of
// lane l is key 32 i + l of that run) with per-bit ballots per warp, per-warp
// digit counts are scanned across the warps, and every key goes to
//   (keys of smaller digits) + (keys of its digit in earlier tiles)
//   + (its rank inside the tile).
// With NEXT, each written key also adds one to its next digit's count in
// the tile it lands in (the next pass's count matrix).  With RECTS (the last
// pass), each key's Gaussian also has its tile rectangle computed (its
// position and radius gathered as soon as its id is loaded, so the latency
// overlaps the ranking) and written beside it: rects[pos], packed 16-bit
// corners, empty when culled.
struct RectOut {
    const float* splat2d;
    const int* radius;
    Geom g;
    uint2* rects;
};

__device__ __forceinline__ uint2 pack_rect(int x0, int x1, int y0, int y1) {
    return make_uint2((uint32_t)x0 | ((uint32_t)x1 << 16), (uint32_t)y0 | ((uint32_t)y1 << 16));
}

template <int SHIFT, int BITS, int NSHIFT, int NBITS, bool NEXT, bool RECTS>
__global__ void __launch_bounds__(kRsThreads)
radix_scatter_kernel(int n, const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                     uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const uint32_t* __restrict__ colpre,
                     const uint32_t* __restrict__ tot, uint32_t* __restrict__ cnext, uint32_t* __restrict__ err,
                     RectOut ro) {
    constexpr int NB = 1 << BITS;
    constexpr int DPT = NB / kRsThreads;  // digits owned by each thread
    __shared__ uint16_t s_w[kRsWarps][NB];
    __shared__ uint32_t s_base[NB];
    __shared__ uint32_t s_wsum[kRsWarps];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = tid; i < kRsWarps * NB / 2; i += kRsThreads) reinterpret_cast<uint32_t*>(&s_w[0][0])[i] = 0u;
    const int tile = blockIdx.x;
    const long long first = (long long)tile * kRsTile + w * 32 * kRsItems + lane;
    uint32_t key[kRsItems], val[kRsItems], rank[kRsItems];
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        const long long idx = first + 32 * i;
        key[i] = idx < n ? kin[idx] : 0xffffffffu;
        val[i] = idx < n ? vin[idx] : 0u;
    }
    uint2 rect[RECTS ? kRsItems : 1];
    if constexpr (RECTS) {
#pragma unroll
        for (int i = 0; i < kRsItems; ++i) {
            int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
            if (first + 32 * i < n) {
                const uint32_t id = val[i];
                if (id >= (uint32_t)n) atomicOr(err, 2u);  // inconsistent counts upstream: nothing is read
                const int r = id < (uint32_t)n ? ro.radius[id] : 0;
                if (r > 0) {
                    const float2 uv = *reinterpret_cast<const float2*>(ro.splat2d + (size_t)id * GSR_REC);
                    tile_rect(uv.x, uv.y, r, ro.g.gx, ro.g.gy, ro.g.twl, ro.g.thl, x0, x1, y0, y1);
                    if (x1 <= x0 || y1 <= y0) x0 = x1 = y0 = y1 = 0;
                }
            }
            rect[i] = pack_rect(x0, x1, y0, y1);
        }
    }
    // digit totals and this tile's column prefixes of the digits d = tid*DPT + j:
    // independent of the ranking, so their loads are issued before it
    uint32_t hv[DPT], cp[DPT];
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
        hv[j] = tot[tid * DPT + j];
        cp[j] = colpre[(size_t)tile * NB + tid * DPT + j];
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        const bool valid = first + 32 * i < n;
        const uint32_t d = (key[i] >> SHIFT) & (NB - 1);
        // A round's 32 digits are usually distinct.  Each lane claims its
        // digit by writing its lane into the counter's spare high bits (a
        // warp holds 256 keys, so a count needs 10 bits) and reads the claim
        // back; only a round where some claim was overwritten compares the
        // digits bit by bit.  The new count clears the claim.
        const uint32_t pre = valid ? s_w[w][d] : 0u;
        __syncwarp();
        if (valid) s_w[w][d] = (uint16_t)(pre | 0x8000u | ((uint32_t)lane << 10));
        __syncwarp();
        const unsigned act = __ballot_sync(kFull, valid);
        const unsigned lost = __ballot_sync(kFull, valid && ((s_w[w][d] >> 10) & 31u) != (uint32_t)lane);
        const unsigned peers = lost ? match_low_bits<BITS>(d, act) : (1u << lane) & act;
        __syncwarp();
        if (valid && lane == 31 - __clz(peers)) s_w[w][d] = (uint16_t)(pre + __popc(peers));
        rank[i] = pre + __popc(peers & lt);
        __syncwarp();
    }
    __syncthreads();
    // digits d = tid*DPT + j: global base and the warps' exclusive offsets
    uint32_t hs = 0;
#pragma unroll
    for (int j = 0; j < DPT; ++j) hs += hv[j];
    uint32_t all = 0;
    uint32_t run = block_excl_scan(hs, s_wsum, &all);
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
        s_base[tid * DPT + j] = run + cp[j];
        run += hv[j];
    }
    // the warps' exclusive offsets, digits strided over the block so that a
    // warp's lanes touch 32 consecutive 16-bit counters
#pragma unroll
    for (int j = 0; j < DPT; ++j) {
        const int d = j * kRsThreads + tid;
        uint32_t wr = 0;
#pragma unroll
        for (int q = 0; q < kRsWarps; ++q) {
            const uint32_t c = s_w[q][d];
            s_w[q][d] = (uint16_t)wr;
            wr += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRsItems; ++i) {
        if (first + 32 * i < n) {
            const uint32_t d = (key[i] >> SHIFT) & (NB - 1);
            const uint32_t pos = s_base[d] + s_w[w][d] + rank[i];
            if (pos >= (uint32_t)n) {  // inconsistent counts: never write outside the buffers
                atomicOr(err, 1u);
                continue;
            }
            kout[pos] = key[i];
            vout[pos] = val[i];
            if (RECTS) ro.rects[pos] = rect[i];
            if (NEXT) {
                constexpr uint32_t NNB = 1u << NBITS;
                atomicAdd(&cnext[(size_t)(pos / kRsTile) * NNB + ((key[i] >> NSHIFT) & (NNB - 1))], 1u);
            }
        }
    }
}

// ---- tile counting sort -----------------------------------------------------
constexpr int kPlaceWarps = 8;
constexpr int kPlaceThreads = 32 * kPlaceWarps;
// Earlier same-row peers a placement lane checks for overlap (more peers:
// every row of the group takes the turn of its rank).
constexpr int kOverlapScan = 8;
constexpr int kMaxWindowTiles = 8192;  // tiles handled per placement window
constexpr int kTargetSMs = 152;
constexpr int kRectPer = 8;                            // Gaussians per thread of the rectangle pass
constexpr int kRectBlock = kRsThreads * kRectPer;      // Gaussians per rectangle block
constexpr int kRectShift = 11;                         // log2(kRectBlock)
static_assert(kRectBlock == 1 << kRectShift, "rectangle block");
// A block's entries stay below 2^16 (its per-tile counts are 16-bit).
constexpr long long kMaxBlockEntries = 65000;

int window_tiles(const Geom& g) { return g.tiles < kMaxWindowTiles ? g.tiles : kMaxWindowTiles; }

// Shared memory of the placement kernel: a 32-bit base per tile and, per
// warp, a 16-bit count per tile (packed two to a word).
size_t place_smem(int tw) { return sizeof(uint32_t) * ((size_t)tw + (size_t)kPlaceWarps * ((tw + 1) / 2)); }

// Number of placement blocks: about one per resident slot of a 152-SM part,
// and enough that no block holds more than kMaxBlockEntries entries.  The
// entries (in depth order, tiles row-major inside each rectangle) are split
// evenly over the blocks' warps, so a block's work does not depend on how
// large its splats are.
int place_blocks(long long cap, const Geom& g) {
    const size_t sm = place_smem(window_tiles(g)) + 1024;
    int per_sm = (int)((size_t)(227 * 1024) / sm);
    per_sm = per_sm < 1 ? 1 : (per_sm > 4 ? 4 : per_sm);
    long long nb = (long long)kTargetSMs * per_sm;
    const long long need = (cap + kMaxBlockEntries - 1) / kMaxBlockEntries;
    return (int)(nb > need ? nb : need);
}

__device__ __forceinline__ void unpack_rect(uint2 r, int& x0, int& x1, int& y0, int& y1) {
    x0 = (int)(r.x & 0xffffu); x1 = (int)(r.x >> 16);
    y0 = (int)(r.y & 0xffffu); y1 = (int)(r.y >> 16);
}

__device__ __forceinline__ uint32_t rect_area(uint2 r) {
    int x0, x1, y0, y1;
    unpack_rect(r, x0, x1, y0, y1);
    return (uint32_t)(x1 - x0) * (uint32_t)(y1 - y0);
}

// Entry counts (rectangle areas) of the depth-ordered Gaussians and their
// exclusive prefix inside each block of 2048; the last block to finish turns
// the block sums into block offsets and stores the entry total in info[4].
// The rectangles come from the last depth-sort pass.
__global__ void __launch_bounds__(kRsThreads)
areas_kernel(int n, const uint2* __restrict__ rects, uint32_t* __restrict__ apre, uint32_t* __restrict__ bsum,
             int nblk, uint32_t* __restrict__ info) {
    __shared__ uint32_t s_wsum[kRsWarps];
    __shared__ bool s_last;
    const int k0 = blockIdx.x * kRectBlock + threadIdx.x * kRectPer;
    uint32_t area[kRectPer], sum = 0;
    if (k0 + kRectPer <= n) {  // a thread's 8 rectangles: 64 contiguous bytes, four 16-byte loads
        const uint4* r4 = reinterpret_cast<const uint4*>(rects + k0);
#pragma unroll
        for (int j = 0; j < kRectPer / 2; ++j) {
            const uint4 q = r4[j];
            area[2 * j] = rect_area(make_uint2(q.x, q.y));
            area[2 * j + 1] = rect_area(make_uint2(q.z, q.w));
        }
    } else {
#pragma unroll
        for (int i = 0; i < kRectPer; ++i) area[i] = k0 + i < n ? rect_area(rects[k0 + i]) : 0u;
    }
#pragma unroll
    for (int i = 0; i < kRectPer; ++i) sum += area[i];
    uint32_t btot;
    uint32_t run = block_excl_scan(sum, s_wsum, &btot);
#pragma unroll
    for (int i = 0; i < kRectPer; ++i) {
        if (k0 + i < n) apre[k0 + i] = run;
        run += area[i];
    }
    if (threadIdx.x == 0) {  // the last block reads only the block sums
        bsum[blockIdx.x] = btot;
        __threadfence();
        s_last = atomicAdd(&info[3], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    uint32_t carry = 0;
    for (int base = 0; base < nblk; base += kRsThreads * 4) {
        const int c0 = base + threadIdx.x * 4;
        uint32_t v[4], s4 = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = c0 + j < nblk ? __ldcg(bsum + c0 + j) : 0u;
            s4 += v[j];
        }
        uint32_t all;
        uint32_t r = carry + block_excl_scan(s4, s_wsum, &all);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (c0 + j < nblk) bsum[c0 + j] = r;
            r += v[j];
        }
        carry += all;
    }
    if (threadIdx.x == 0) info[4] = carry;
}

// Entry prefix of depth-ordered Gaussian k (bsum already holds offsets).
__device__ __forceinline__ uint32_t entry_prefix(const uint32_t* __restrict__ apre, const uint32_t* __restrict__ boff,
                                                 int k) {
    return boff[k >> kRectShift] + apre[k];
}

__device__ __forceinline__ uint32_t warp_entries(uint32_t total, int nwarps) {
    const uint32_t ew = (uint32_t)(((unsigned long long)total + nwarps - 1) / nwarps);
    return ew > 0 ? ew : 1u;
}

// The Gaussian that holds entry e: the last k whose entry prefix is <= e
// (the prefixes do not decrease with k, and a Gaussian with no entries
// shares its prefix with the next one, so the last is the holder).  The warp
// probes 32 points per step, first over the rectangle blocks' offsets, then
// inside the block.
__device__ __forceinline__ int entry_owner(int n, int nblk, const uint32_t* __restrict__ apre,
                                           const uint32_t* __restrict__ boff, uint32_t e, int lane) {
    int lo = 0, hi = nblk;  // boff[lo] <= e throughout (boff[0] = 0)
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) / 32;
        const int p = lo + lane * step;
        const unsigned ok = __ballot_sync(kFull, p < hi && boff[p] <= e);
        lo += (31 - __clz(ok)) * step;
        hi = min(hi, lo + step);
    }
    const uint32_t r = e - boff[lo];
    int klo = lo << kRectShift;  // apre[klo] = 0 <= r throughout
    int khi = min(n, klo + kRectBlock);
    while (khi - klo > 1) {
        const int step = (khi - klo + 31) / 32;
        const int p = klo + lane * step;
        const unsigned ok = __ballot_sync(kFull, p < khi && apre[p] <= r);
        klo += (31 - __clz(ok)) * step;
        khi = min(khi, klo + step);
    }
    return klo;
}

// Per-warp staging of 32 consecutive depth-ordered Gaussians: their
// rectangles, the exclusive prefixes of their entry counts (areas) and of
// their row counts (rectangle heights), ids and depth keys.  Work is handed
// to lanes one rectangle row at a time: row unit u of the batch belongs to
// the last Gaussian whose row prefix is <= u.
struct WarpBatch {
    uint32_t pre[32];    // entries before Gaussian j in the batch
    uint32_t rpre[33];   // rows before Gaussian j; rpre[32] = rows of the batch
    int x0[32], wd[32], y0[32];
    uint32_t id[32], dk[32];
};

// Fills the warp's batch (lane = Gaussian k, absent at k >= n); returns the
// batch's entry count (and its row count in *rows).
__device__ __forceinline__ uint32_t stage_batch(WarpBatch& wb, int lane, bool present, uint2 pr, uint32_t id,
                                                uint32_t dk, uint32_t* rows) {
    int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
    if (present) unpack_rect(pr, x0, x1, y0, y1);
    const int wd = x1 - x0;
    const uint32_t ht = wd > 0 ? (uint32_t)(y1 - y0) : 0u;
    const uint32_t area = (uint32_t)wd * ht;
    uint32_t inc = area, rinc = ht;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, inc, o);
        const uint32_t r = __shfl_up_sync(kFull, rinc, o);
        if (lane >= o) {
            inc += t;
            rinc += r;
        }
    }
    wb.pre[lane] = inc - area;
    wb.rpre[lane] = rinc - ht;
    if (lane == 31) wb.rpre[32] = rinc;
    wb.x0[lane] = x0;
    wb.wd[lane] = wd;
    wb.y0[lane] = y0;
    wb.id[lane] = id;
    wb.dk[lane] = dk;
    *rows = __shfl_sync(kFull, rinc, 31);
    return __shfl_sync(kFull, inc, 31);
}

// One rectangle row handed to a lane: tiles row_t0 + x for x in [xs, xe)
// (window-relative tile ids), of Gaussian lane j of the batch, tile row y.
struct RowWork {
    int j, y, row_t0, xs, xe;
};

// Row unit u of the batch, clipped to the warp's entries [e0, e1) (pk =
// global index of the batch's first entry).  Returns false when nothing of
// the row lies in the range.
__device__ __forceinline__ bool row_unit(const WarpBatch& wb, uint32_t u, uint32_t pk, uint32_t e0, uint32_t e1,
                                         const Geom& g, int t0, RowWork& r) {
    int lo = 0, hi = 31;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int mid = (lo + hi + 1) >> 1;
        if (wb.rpre[mid] <= u) lo = mid; else hi = mid - 1;
    }
    const int ri = (int)(u - wb.rpre[lo]);
    const int wd = wb.wd[lo];
    const uint32_t gp = pk + wb.pre[lo] + (uint32_t)(ri * wd);  // global index of the row's first entry
    const int xs = e0 > gp ? (int)(e0 - gp) : 0;
    const int xe = e1 - gp < (uint32_t)wd ? (int)(e1 - gp) : wd;
    if (gp >= e1 || xe <= xs) return false;
    r.j = lo;
    r.y = wb.y0[lo] + ri;
    r.row_t0 = r.y * g.gx + wb.x0[lo] - t0;
    r.xs = xs;
    r.xe = xe;
    return true;
}

// Walks the entries [e0, e1) of one warp in depth order, 32 Gaussians at a
// time and 32 rectangle rows per round: f(ok, row) on every lane of every
// round (ok false when the lane has no row), so f may use warp intrinsics.
template <bool IDS, class F>
__device__ __forceinline__ void walk_rows(WarpBatch& wb, int lane, int n, uint32_t e0, uint32_t e1, int k,
                                          const uint2* __restrict__ rects, const uint32_t* __restrict__ order,
                                          const uint32_t* __restrict__ dkeys, uint32_t pk, const Geom& g, int t0,
                                          F&& f) {
    while (pk < e1 && k < n) {
        const int kk = k + lane;
        const bool present = kk < n;
        uint32_t br;
        const uint32_t bt = stage_batch(wb, lane, present, present ? rects[kk] : make_uint2(0u, 0u),
                                        IDS && present ? order[kk] : 0u, IDS && dkeys && present ? dkeys[kk] : 0u,
                                        &br);
        __syncwarp();
        for (uint32_t base = 0; base < br; base += 32) {
            const uint32_t u = base + lane;
            RowWork r;
            const bool ok = u < br && row_unit(wb, u, pk, e0, e1, g, t0, r);
            f(ok, r);
        }
        __syncwarp();
        pk += bt;
        k += 32;
    }
}

// Window of the entry counts: tile columns [c0, c0 + cw) x rows [r0, r0 + rh),
// cw * rh <= kMaxWindowTiles.
struct CountWindow {
    int c0, cw, r0, rh;
};

// Adds the tile rectangle [x0, x1) x [y0, y1), clipped to the window, to the
// window's 2D difference array d (row-major, cw wide): +1 at its first
// corner and one past its last, -1 at the other two; corners past the
// window's right or bottom edge change no counted cell and are left out.
__device__ __forceinline__ void diff_rect(int* d, const CountWindow& cwin, int x0, int x1, int y0, int y1) {
    x0 = max(x0 - cwin.c0, 0); x1 = min(x1 - cwin.c0, cwin.cw);
    y0 = max(y0 - cwin.r0, 0); y1 = min(y1 - cwin.r0, cwin.rh);
    if (x0 >= x1 || y0 >= y1) return;
    atomicAdd(&d[y0 * cwin.cw + x0], 1);
    if (x1 < cwin.cw) atomicAdd(&d[y0 * cwin.cw + x1], -1);
    if (y1 < cwin.rh) {
        atomicAdd(&d[y1 * cwin.cw + x0], -1);
        if (x1 < cwin.cw) atomicAdd(&d[y1 * cwin.cw + x1], 1);
    }
}

// Counts, per placement block, the entries of every tile in a window:
// m[b][tile].  A warp takes its slice's Gaussians 32 at a time, one per
// lane, and adds each one's entries as rectangles to a 2D difference array
// of the window (a Gaussian that straddles a slice boundary keeps the tail
// of one row, whole rows and the head of another: up to three rectangles);
// prefix sums along the rows and then down the columns turn it into the
// counts.
__global__ void __launch_bounds__(kPlaceThreads)
chunk_hist_kernel(int n, int nb, int nblk, Geom g, CountWindow cwin, const uint2* __restrict__ rects,
                  const uint32_t* __restrict__ apre, const uint32_t* __restrict__ boff,
                  uint32_t* __restrict__ wstart, const uint32_t* __restrict__ info, uint32_t* __restrict__ m) {
    extern __shared__ int d[];  // [rh][cw]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cells = cwin.cw * cwin.rh;
    for (int q = threadIdx.x; q < cells; q += kPlaceThreads) d[q] = 0;
    __syncthreads();
    const int b = blockIdx.x;
    const uint32_t total = info[4];
    const uint32_t ew = warp_entries(total, nb * kPlaceWarps);
    const unsigned long long e0l = (unsigned long long)(b * kPlaceWarps + w) * ew;
    if (e0l < total) {
        const uint32_t e0 = (uint32_t)e0l;
        const int kw = entry_owner(n, nblk, apre, boff, e0, lane);  // also the placement warp's start
        if (lane == 0) wstart[b * kPlaceWarps + w] = (uint32_t)kw;
        const uint32_t e1 = total - e0 < ew ? total : e0 + ew;
        for (int k = kw; k < n; k += 32) {
            const int kk = k + lane;
            uint32_t p = 0xffffffffu;
            int x0 = 0, x1 = 0, y0 = 0, y1 = 0;
            if (kk < n) {
                p = entry_prefix(apre, boff, kk);
                unpack_rect(rects[kk], x0, x1, y0, y1);
            }
            if (__ballot_sync(kFull, p < e1) == 0u) break;  // prefixes increase with k
            const uint32_t wd = (uint32_t)(x1 - x0), area = wd * (uint32_t)(y1 - y0);
            if (p >= e1 || area == 0u || p + area <= e0) continue;
            const uint32_t a = e0 > p ? e0 - p : 0u;
            const uint32_t z = e1 - p < area ? e1 - p : area;  // entries [a, z) of this Gaussian are the slice's
            if (a == 0u && z == area) {
                diff_rect(d, cwin, x0, x1, y0, y1);
                continue;
            }
            const int ra = (int)(a / wd), ca = (int)(a % wd), rz = (int)(z / wd), cz = (int)(z % wd);
            if (ra == rz) {
                diff_rect(d, cwin, x0 + ca, x0 + cz, y0 + ra, y0 + ra + 1);
                continue;
            }
            int rf = ra;
            if (ca > 0) {
                diff_rect(d, cwin, x0 + ca, x1, y0 + ra, y0 + ra + 1);
                rf = ra + 1;
            }
            if (rz > rf) diff_rect(d, cwin, x0, x1, y0 + rf, y0 + rz);
            if (cz > 0) diff_rect(d, cwin, x0, x0 + cz, y0 + rz, y0 + rz + 1);
        }
    }
    __syncthreads();
    // prefix sums along each row (a warp per row, 32 cells at a time) ...
    for (int y = w; y < cwin.rh; y += kPlaceWarps) {
        int carry = 0;
        for (int x = 0; x < cwin.cw; x += 32) {
            const int i = y * cwin.cw + x + lane;
            int v = x + lane < cwin.cw ? d[i] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(kFull, v, o);
                if (lane >= o) v += u;
            }
            v += carry;
            if (x + lane < cwin.cw) d[i] = v;
            carry = __shfl_sync(kFull, v, 31);
        }
    }
    __syncthreads();
    // ... then down each column, written out as the block's counts
    for (int x = threadIdx.x; x < cwin.cw; x += kPlaceThreads) {
        int run = 0;
        size_t o = (size_t)b * g.tiles + (size_t)cwin.r0 * g.gx + cwin.c0 + x;
        for (int y = 0; y < cwin.rh; ++y, o += g.gx) {
            run += d[y * cwin.cw + x];
            m[o] = (uint32_t)run;
        }
    }
}

// Writes the entries of the tiles in the window: block b's entries of tile
// t start at start[t] + m[b][t] (m already column-scanned); each warp owns a
// consecutive slice of the block's entries, and its per-tile offsets come
// from the warps before it.  Rows of one tile row in the same round of 32
// are ranked by lane with a match mask on the row index, and overlapping
// ones take turns, so every tile receives its entries in depth order.
template <bool KEYS>
__global__ void __launch_bounds__(kPlaceThreads)
place_kernel(int n, int nb, Geom g, int t0, int tw, uint32_t cap, const uint32_t* __restrict__ order,
             const uint32_t* __restrict__ dkeys, const uint2* __restrict__ rects, const uint32_t* __restrict__ apre,
             const uint32_t* __restrict__ boff, const uint32_t* __restrict__ wstart,
             const uint32_t* __restrict__ info, const uint32_t* __restrict__ m, const uint32_t* __restrict__ start,
             uint32_t* __restrict__ point_list, uint64_t* __restrict__ keys_out) {
    extern __shared__ uint32_t sm[];
    __shared__ WarpBatch s_wb[kPlaceWarps];
    // over capacity or inconsistent counts: nothing is placed (the ranges are empty)
    if (info[0] > cap || info[1] || info[0] != info[4]) return;
    const int tw2 = (tw + 1) / 2;
    uint32_t* s_base = sm;
    uint32_t* s_cnt = sm + tw;  // [kPlaceWarps][tw2] packed 16-bit counts
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int i = tid; i < kPlaceWarps * tw2; i += kPlaceThreads) s_cnt[i] = 0;
    const int b = blockIdx.x;
    const uint32_t total = info[4];
    const uint32_t ew = warp_entries(total, nb * kPlaceWarps);
    const unsigned long long e0l = (unsigned long long)(b * kPlaceWarps + w) * ew;
    const int kw = e0l < total ? (int)wstart[b * kPlaceWarps + w] : n;
    const bool mine = e0l < total && (unsigned)kw < (unsigned)n;
    const uint32_t e0 = mine ? (uint32_t)e0l : 0u;
    const uint32_t e1 = !mine ? 0u : (total - e0 < ew ? total : e0 + ew);
    const int k = mine ? kw : 0;
    const uint32_t pk = mine ? entry_prefix(apre, boff, k) : 0u;
    WarpBatch& wb = s_wb[w];
    uint32_t* wc = s_cnt + (size_t)w * tw2;
    __syncthreads();
    // per-warp entry counts of each tile
    if (mine)
        walk_rows<false>(wb, lane, n, e0, e1, k, rects, nullptr, nullptr, pk, g, t0, [&](bool ok, const RowWork& r) {
            if (!ok) return;
            const int lo = max(r.row_t0 + r.xs, 0), hi = min(r.row_t0 + r.xe, tw);
            for (int q = lo >> 1; 2 * q < hi; ++q)
                atomicAdd(&wc[q], (2 * q >= lo ? 1u : 0u) + (2 * q + 1 < hi ? 0x10000u : 0u));
        });
    __syncthreads();
    // tile bases; per-warp exclusive offsets (two tiles per word)
    for (int q = tid; q < tw2; q += kPlaceThreads) {
        const int t = 2 * q;
        const size_t mb = (size_t)b * g.tiles + t0;
        s_base[t] = m[mb + t] + start[t0 + t];
        if (t + 1 < tw) s_base[t + 1] = m[mb + t + 1] + start[t0 + t + 1];
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int v = 0; v < kPlaceWarps; ++v) {
            const uint32_t x = s_cnt[(size_t)v * tw2 + q];
            s_cnt[(size_t)v * tw2 + q] = lo | (hi << 16);
            lo += x & 0xffffu;
            hi += x >> 16;
        }
    }
    __syncthreads();
    if (!mine) return;
    uint16_t* c16 = reinterpret_cast<uint16_t*>(wc);
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t key_total = info[0];
    walk_rows<true>(wb, lane, n, e0, e1, k, rects, order, KEYS ? dkeys : nullptr, pk, g, t0,
                    [&](bool ok, const RowWork& r) {
        // rows of the same tile row in one round may share tiles: those
        // take turns in lane order (lane order is depth order).  A row that
        // overlaps no earlier row of its tile row goes in the first turn,
        // the others in the turn of their rank; rows of different tile
        // rows never share a tile.
        const unsigned peers = __match_any_sync(kFull, ok ? (uint32_t)r.y : 0xffffffffu);
        const int rank = __popc(peers & lt);
        const int maxrank = __reduce_max_sync(kFull, ok ? rank : 0);
        int my_turn = rank;
        if (maxrank > 0 && maxrank <= kOverlapScan) {
            const int ts = ok ? r.row_t0 + r.xs : 0, te = ok ? r.row_t0 + r.xe : 0;
            unsigned below = ok ? (peers & lt) : 0u;
            bool overlap = false;
            for (int q = 0; q < maxrank; ++q) {  // earlier peers, nearest first
                const int pl = below ? 31 - __clz(below) : lane;
                if (below) below ^= 1u << pl;
                const int ps = __shfl_sync(kFull, ts, pl), pe = __shfl_sync(kFull, te, pl);
                overlap |= pl != lane && ps < te && ts < pe;
            }
            if (!overlap) my_turn = 0;
        }
        const int turns = __reduce_max_sync(kFull, ok ? my_turn + 1 : 0);
        const uint32_t id = ok ? wb.id[r.j] : 0u;
        const uint64_t dk = KEYS && ok ? (uint64_t)wb.dk[r.j] : 0ull;
        for (int turn = 0; turn < turns; ++turn) {
            if (ok && my_turn == turn) {
                for (int xb = r.xs; xb < r.xe; xb += 4) {
                    int t[4];
                    bool in[4];
                    uint32_t c[4], sb[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        t[i] = r.row_t0 + xb + i;
                        in[i] = xb + i < r.xe && (unsigned)t[i] < (unsigned)tw;
                        c[i] = in[i] ? (uint32_t)c16[t[i]] : 0u;
                        sb[i] = in[i] ? s_base[t[i]] : 0u;
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (!in[i]) continue;
                        const uint32_t pos = sb[i] + c[i];
                        if (pos < key_total) {  // always, unless the counts were inconsistent
                            point_list[pos] = id;
                            if (KEYS) keys_out[pos] = ((uint64_t)(uint32_t)(t[i] + t0) << 32) | dk;
                        }
                        c16[t[i]] = (uint16_t)(c[i] + 1);
                    }
                }
            }
            __syncwarp();
        }
    });
}

// ---- scratch ------------------------------------------------------------------
struct BinScratch {
    uint32_t *ka, *va, *kb, *vb;   // [n] ping-pong keys / values of the depth sort
    uint32_t *c0, *c1, *c2;        // [rs_tiles][digits] count matrices of the three passes
    uint32_t *t0, *t1, *t2;        // digit totals
    uint32_t* info;                // [8]: key total, sort error flag, finished colscan blocks,
                                   //      finished rectangle blocks, entry total
    uint2* rects;                  // [n] packed tile rectangles in depth order
    uint32_t* apre;                // [n] entry prefix inside each rectangle block
    uint32_t* bsum;                // [n / 2048] rectangle block sums, then offsets
    uint32_t* wstart;              // [nb * warps] first Gaussian of each placement warp
    uint32_t* m;                   // [nb][tiles] block x tile counts, then bases
    uint32_t *ttot, *tstart;       // [tiles]
    int nb;                        // placement blocks
    size_t zero_bytes;             // c1 .. info are zeroed together
    size_t total;
};

int rect_blocks(int n) { return (n + kRectBlock - 1) / kRectBlock; }

void bin_layout(int n, const Geom& g, long long cap, char* base, BinScratch& s) {
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const size_t rt = (size_t)(rs_tiles(n) > 0 ? rs_tiles(n) : 1);
    s.nb = place_blocks(cap, g);
    const size_t nb = (size_t)s.nb;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return base ? base + o : nullptr; };
    s.ka = (uint32_t*)take(4 * nn);
    s.va = (uint32_t*)take(4 * nn);
    s.kb = (uint32_t*)take(4 * nn);
    s.vb = (uint32_t*)take(4 * nn);
    s.c0 = (uint32_t*)take(4 * rt * (1u << kRsB0));
    s.t0 = (uint32_t*)take(4 * (1u << kRsB0));
    s.t1 = (uint32_t*)take(4 * (1u << kRsB1));
    s.t2 = (uint32_t*)take(4 * (1u << kRsB2));
    const size_t z0 = off;
    s.c1 = (uint32_t*)take(4 * rt * (1u << kRsB1));
    s.c2 = (uint32_t*)take(4 * rt * (1u << kRsB2));
    s.info = (uint32_t*)take(32);
    s.zero_bytes = off - z0;
    s.rects = (uint2*)take(8 * nn);
    s.apre = (uint32_t*)take(4 * nn);
    s.bsum = (uint32_t*)take(4 * (size_t)(rect_blocks(n) > 0 ? rect_blocks(n) : 1));
    s.wstart = (uint32_t*)take(4 * nb * kPlaceWarps);
    s.m = (uint32_t*)take(4 * nb * (size_t)g.tiles);
    s.ttot = (uint32_t*)take(4 * (size_t)g.tiles);
    s.tstart = (uint32_t*)take(4 * (size_t)g.tiles);
    s.total = off;
}

int colscan(int rows, int cols, uint32_t* m, uint32_t* tot, uint32_t* start, uint32_t* ranges, uint32_t* info,
            cudaStream_t st, uint32_t cap = 0xffffffffu, uint32_t* count_out = nullptr, uint32_t* order = nullptr) {
    static_assert(kOrderThreads == 1024, "the column scan's last block computes the tile order");
    colscan_kernel<<<(cols + 31) / 32, 1024, 0, st>>>(rows, cols, m, tot, start, ranges, info, cap, count_out,
                                                      order);
    return check_launch();
}

// The longest-first tile order alone (a view without Gaussians).
__global__ void __launch_bounds__(kOrderThreads)
order_kernel(int tiles, const uint2* __restrict__ ranges, uint32_t* __restrict__ order) {
    __shared__ uint32_t cnt[kOrderBuckets];
    tile_order_block(tiles, ranges, order, cnt);
}

int smem_optin(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return GSR_OK;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return e == cudaSuccess ? GSR_OK : cuda_fail(e);
}

}  // namespace
}  // namespace gsr

using namespace gsr;

extern "C" int gsr_bin_scratch_bytes(int32_t n, int32_t width, int32_t height, int32_t tile_w,
                                     int32_t tile_h, int64_t key_capacity, size_t* bytes) {
    Geom g;
    if (n < 0 || key_capacity < 0 || key_capacity >= 0xffffffffll || !bytes ||
        !make_geom(width, height, tile_w, tile_h, g))
        return GSR_EINVAL;
    BinScratch s;
    bin_layout(n, g, key_capacity, nullptr, s);
    *bytes = s.total;
    return GSR_OK;
}

namespace gsr {
namespace {

// count_dev == nullptr: synchronous (reads the key count, *n_keys);
// otherwise the count and status go to count_dev and nothing waits.
int bin_sort_impl(int32_t n, int32_t width, int32_t height, int32_t tile_w, int32_t tile_h, const float* splat2d,
                  const int32_t* radius, int64_t key_capacity, void* scratch, size_t scratch_bytes,
                  uint32_t* point_list, uint32_t* tile_ranges, uint64_t* keys_out, int64_t* n_keys,
                  uint32_t* count_dev, uint32_t* tile_order, gsr_stream_t stream_) {
    Geom g;
    if (n < 0 || key_capacity < 0 || key_capacity >= 0xffffffffll || (!n_keys && !count_dev) ||
        !make_geom(width, height, tile_w, tile_h, g))
        return GSR_EINVAL;
    if (!tile_ranges || !scratch || (n > 0 && (!splat2d || !radius)) || (key_capacity > 0 && !point_list))
        return GSR_EINVAL;
    if (!aligned16(splat2d) || !aligned16(scratch) || (keys_out && !aligned8(keys_out))) return GSR_EINVAL;
    cudaStream_t st = (cudaStream_t)stream_;
    BinScratch s;
    bin_layout(n, g, key_capacity, (char*)scratch, s);
    if (scratch_bytes < s.total) return GSR_ESCRATCH;
    if (n_keys) *n_keys = 0;
    int rc;
    cudaError_t e;
    if (n == 0) {
        e = cudaMemsetAsync(tile_ranges, 0, sizeof(uint32_t) * 2 * (size_t)g.tiles, st);
        if (e == cudaSuccess && count_dev) e = cudaMemsetAsync(count_dev, 0, 2 * sizeof(uint32_t), st);
        if (e != cudaSuccess) return cuda_fail(e);
        if (tile_order) {  // every list empty: the order of the (empty) ranges
            order_kernel<<<1, kOrderThreads, 0, st>>>(g.tiles, reinterpret_cast<const uint2*>(tile_ranges),
                                                      tile_order);
            return check_launch();
        }
        return GSR_OK;
    }
    e = cudaMemsetAsync(s.c1, 0, s.zero_bytes, st);
    if (e != cudaSuccess) return cuda_fail(e);

    // 1. (depth, id) order: keys + first-digit counts, then three passes
    const int rt = rs_tiles(n);
    depth_keys_kernel<<<rt, kRsThreads, 0, st>>>(n, splat2d, radius, s.ka, s.va, s.c0);
    if ((rc = check_launch()) != GSR_OK) return rc;
    if ((rc = colscan(rt, 1 << kRsB0, s.c0, s.t0, nullptr, nullptr, nullptr, st)) != GSR_OK) return rc;
    const RectOut no_rects = {nullptr, nullptr, g, nullptr};
    radix_scatter_kernel<0, kRsB0, kRsS1, kRsB1, true, false><<<rt, kRsThreads, 0, st>>>(
        n, s.ka, s.va, s.kb, s.vb, s.c0, s.t0, s.c1, s.info + 1, no_rects);
    if ((rc = check_launch()) != GSR_OK) return rc;
    if ((rc = colscan(rt, 1 << kRsB1, s.c1, s.t1, nullptr, nullptr, nullptr, st)) != GSR_OK) return rc;
    radix_scatter_kernel<kRsS1, kRsB1, kRsS2, kRsB2, true, false><<<rt, kRsThreads, 0, st>>>(
        n, s.kb, s.vb, s.ka, s.va, s.c1, s.t1, s.c2, s.info + 1, no_rects);
    if ((rc = check_launch()) != GSR_OK) return rc;
    if ((rc = colscan(rt, 1 << kRsB2, s.c2, s.t2, nullptr, nullptr, nullptr, st)) != GSR_OK) return rc;
    // the last pass also writes each Gaussian's tile rectangle in depth order
    radix_scatter_kernel<kRsS2, kRsB2, 0, 1, false, true><<<rt, kRsThreads, 0, st>>>(
        n, s.ka, s.va, s.kb, s.vb, s.c2, s.t2, nullptr, s.info + 1, RectOut{splat2d, radius, g, s.rects});
    if ((rc = check_launch()) != GSR_OK) return rc;
    const uint32_t* order = s.vb;
    const uint32_t* dkeys = s.kb;

    // 2. entry prefixes in depth order; per block x tile counts (which also
    //    find the first Gaussian of every placement warp); column scan, tile
    //    starts and ranges
    const int nr = rect_blocks(n);
    areas_kernel<<<nr, kRsThreads, 0, st>>>(n, s.rects, s.apre, s.bsum, nr, s.info);
    if ((rc = check_launch()) != GSR_OK) return rc;
    const int tw = window_tiles(g);
    {   // count windows: whole tile rows (row pieces when a row is longer than a window)
        CountWindow cwin;
        cwin.cw = g.gx < kMaxWindowTiles ? g.gx : kMaxWindowTiles;
        const int rows = kMaxWindowTiles / cwin.cw;
        const size_t hsm = sizeof(int) * (size_t)cwin.cw * (size_t)(rows < g.gy ? rows : g.gy);
        if ((rc = smem_optin((const void*)chunk_hist_kernel, hsm)) != GSR_OK) return rc;
        for (cwin.r0 = 0; cwin.r0 < g.gy; cwin.r0 += rows) {
            cwin.rh = g.gy - cwin.r0 < rows ? g.gy - cwin.r0 : rows;
            for (int c0 = 0; c0 < g.gx; c0 += kMaxWindowTiles) {
                cwin.c0 = c0;
                cwin.cw = g.gx - c0 < kMaxWindowTiles ? g.gx - c0 : kMaxWindowTiles;
                chunk_hist_kernel<<<s.nb, kPlaceThreads, hsm, st>>>(n, s.nb, nr, g, cwin, s.rects, s.apre,
                                                                    s.bsum, s.wstart, s.info, s.m);
                if ((rc = check_launch()) != GSR_OK) return rc;
            }
        }
    }
    const uint32_t cap = (uint32_t)key_capacity;
    if ((rc = colscan(s.nb, g.tiles, s.m, s.ttot, s.tstart, tile_ranges, s.info, st, cap, count_dev, tile_order)) !=
        GSR_OK)
        return rc;
    if (count_dev) {  // placement checks the count on the device
        const size_t psm = place_smem(tw);
        auto pk = keys_out ? place_kernel<true> : place_kernel<false>;
        if ((rc = smem_optin((const void*)pk, psm)) != GSR_OK) return rc;
        for (int t0 = 0; t0 < g.tiles; t0 += tw) {
            const int wt = g.tiles - t0 < tw ? g.tiles - t0 : tw;
            pk<<<s.nb, kPlaceThreads, psm, st>>>(n, s.nb, g, t0, wt, cap, order, dkeys, s.rects, s.apre, s.bsum,
                                                 s.wstart, s.info, s.m, s.tstart, point_list, keys_out);
            if ((rc = check_launch()) != GSR_OK) return rc;
        }
        return GSR_OK;
    }
    uint32_t info[5] = {0, 0, 0, 0, 0};
    e = cudaMemcpyAsync(info, s.info, sizeof(info), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    // a sort pass found inconsistent counts, or the two entry totals differ (not expected)
    if (info[1] || info[0] != info[4]) return GSR_ECUDA;
    const uint32_t total = info[0];
    *n_keys = (int64_t)total;
    if ((long long)total > key_capacity) return GSR_ECAPACITY;
    if (total == 0) return GSR_OK;

    // 3. entries written in place
    const size_t psm = place_smem(tw);
    auto pk = keys_out ? place_kernel<true> : place_kernel<false>;
    if ((rc = smem_optin((const void*)pk, psm)) != GSR_OK) return rc;
    for (int t0 = 0; t0 < g.tiles; t0 += tw) {
        const int wt = g.tiles - t0 < tw ? g.tiles - t0 : tw;
        pk<<<s.nb, kPlaceThreads, psm, st>>>(n, s.nb, g, t0, wt, cap, order, dkeys, s.rects, s.apre, s.bsum,
                                             s.wstart, s.info, s.m, s.tstart, point_list, keys_out);
        if ((rc = check_launch()) != GSR_OK) return rc;
    }
    return GSR_OK;
}

}  // namespace
}  // namespace gsr

extern "C" int gsr_bin_sort(int32_t n, int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                            const float* splat2d, const int32_t* radius, int64_t key_capacity,
                            void* scratch, size_t scratch_bytes, uint32_t* point_list,
                            uint32_t* tile_ranges, uint64_t* keys_out, int64_t* n_keys,
                            gsr_stream_t stream) {
    if (!n_keys) return GSR_EINVAL;
    return bin_sort_impl(n, width, height, tile_w, tile_h, splat2d, radius, key_capacity, scratch, scratch_bytes,
                         point_list, tile_ranges, keys_out, n_keys, nullptr, nullptr, stream);
}

extern "C" int gsr_bin_sort_async(int32_t n, int32_t width, int32_t height, int32_t tile_w, int32_t tile_h,
                                  const float* splat2d, const int32_t* radius, int64_t key_capacity,
                                  void* scratch, size_t scratch_bytes, uint32_t* point_list,
                                  uint32_t* tile_ranges, uint64_t* keys_out, uint32_t* count_dev,
                                  uint32_t* tile_order, gsr_stream_t stream) {
    if (!count_dev) return GSR_EINVAL;
    return bin_sort_impl(n, width, height, tile_w, tile_h, splat2d, radius, key_capacity, scratch, scratch_bytes,
                         point_list, tile_ranges, keys_out, nullptr, count_dev, tile_order, stream);
}
