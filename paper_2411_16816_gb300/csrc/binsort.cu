// binsort.cu -- tile duplication and sorting (paper Sec. 3.2 "Projection, tiling, and
// sorting": Gaussians are duplicated into every tile they intersect and sorted by
// depth; Sec. 3.3 / App. A.1: lidar Gaussians sorted by range, azimuth tile ids wrapped
// into [0, M_phi) before the identifier is formed).
//
// Order of the lists: (global tile, depth, Gaussian index).  It is produced in two
// stable stages instead of one 48-bit key sort:
//   1. compact the visible (sensor, Gaussian) pairs and radix-sort them by the FP32 bit
//      pattern of their depth (32-bit key, stable, so equal depths keep index order);
//   2. emit every pair's tiles in that depth order and stable radix-sort the
//      intersections by tile id only (16 bits for a 6-camera + lidar frame).
// Stage 2 touches each intersection in ceil(bits(tiles)/8) passes instead of six.
//
// Every device-wide step is reduce -> scan -> apply with no inter-block waiting, so
// nothing in this file can spin.  Counts that only the device knows (visible pairs,
// intersections) are read by the kernels from device memory; grids are sized from host
// upper bounds and surplus blocks do no work.
#include "status.cuh"
#include "types.cuh"

namespace splat {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // 2048
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 2048

__device__ __forceinline__ int64_t eff_count(const int64_t* count_ptr, int64_t max_count, int64_t capacity) {
    if (!count_ptr) return max_count;
    const int64_t c = *count_ptr;
    if (c > capacity) return 0;  // over capacity: the lists are invalid, touch nothing
    return c < max_count ? c : max_count;
}

// Exclusive scan of one value per thread across a 256-thread block.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total, int64_t* sm /*[9]*/) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int w = 0; w < kScanThreads / 32; w++) {
            const int64_t t = sm[w];
            sm[w] = run;
            run += t;
        }
        sm[8] = run;
    }
    __syncthreads();
    const int64_t res = x - v + sm[warp];
    if (total) *total = sm[8];
    __syncthreads();
    return res;
}

// Contiguous 32-bit inputs and outputs take two 16-byte accesses per thread.
__device__ __forceinline__ void ld8_u32(const void* p, int64_t i, uint32_t (&u)[8]) {
    const uint4* q = reinterpret_cast<const uint4*>(reinterpret_cast<const uint32_t*>(p) + i);
    const uint4 a = q[0], b = q[1];
    u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
    u[4] = b.x; u[5] = b.y; u[6] = b.z; u[7] = b.w;
}
__host__ __device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// A thread's kScanItems consecutive items: two 16-byte loads when the input is a
// contiguous 32-bit array aligned for them (In::kVec and in.vec) and all are in range.
template <typename In>
__device__ __forceinline__ void load_items(const In& in, int64_t base, int64_t count, int64_t (&v)[kScanItems]) {
    if constexpr (In::kVec) {
        if (in.vec && base + kScanItems <= count) {
            in.load8(base, v);
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < kScanItems; k++) v[k] = base + k < count ? in(base + k) : 0;
}

template <typename In>
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(In in, int64_t max_count, const int64_t* count_ptr,
                                                              int64_t capacity, int64_t* partials) {
    __shared__ int64_t sm[9];
    const int64_t count = eff_count(count_ptr, max_count, capacity);
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    if ((int64_t)blockIdx.x * kScanTile >= count) {   // an empty block (the grid is an upper bound)
        if (threadIdx.x == 0) partials[blockIdx.x] = 0;
        return;
    }
    int64_t v[kScanItems];
    load_items(in, base, count, v);
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) s += v[k];
    int64_t total;
    block_exclusive_scan(s, &total, sm);
    if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

// Single block: exclusive scan of the partials of the blocks that hold items, in place;
// writes the grand total.
__global__ void __launch_bounds__(1024) k_scan_top(int64_t* partials, int64_t nparts, int64_t* total,
                                                   int64_t max_count, const int64_t* count_ptr, int64_t capacity) {
    __shared__ int64_t sm[33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t active = (eff_count(count_ptr, max_count, capacity) + kScanTile - 1) / kScanTile;
    if (active < nparts) nparts = active;
    int64_t carry = 0;
    for (int64_t base = 0; base < nparts; base += 1024) {
        const int64_t idx = base + threadIdx.x;
        const int64_t v = idx < nparts ? partials[idx] : 0;
        int64_t x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sm[warp] = x;
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t run = 0;
            for (int w = 0; w < 32; w++) {
                const int64_t t = sm[w];
                sm[w] = run;
                run += t;
            }
            sm[32] = run;
        }
        __syncthreads();
        if (idx < nparts) partials[idx] = carry + x - v + sm[warp];
        carry += sm[32];
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

template <typename In, typename Out>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(In in, Out out, int64_t max_count,
                                                             const int64_t* count_ptr, int64_t capacity,
                                                             const int64_t* partials) {
    __shared__ int64_t sm[9];
    const int64_t count = eff_count(count_ptr, max_count, capacity);
    if ((int64_t)blockIdx.x * kScanTile >= count) return;   // an empty block (uniform)
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    load_items(in, base, count, v);
    int64_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) s += v[k];
    int64_t run = block_exclusive_scan(s, nullptr, sm) + partials[blockIdx.x];
    if constexpr (Out::kVec) {
        if (out.vec && base + kScanItems <= count) {
            int64_t pre[kScanItems];
#pragma unroll
            for (int k = 0; k < kScanItems; k++) {
                pre[k] = run;
                run += v[k];
            }
            out.store8(base, pre);
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        if (base + k < count) out(base + k, run, v[k]);
        run += v[k];
    }
}

template <typename In, typename Out>
void device_scan(In in, Out out, int64_t max_count, const int64_t* count_ptr, int64_t capacity, int64_t* partials,
                 int64_t* total, cudaStream_t st) {
    const int64_t nblocks = (max_count + kScanTile - 1) / kScanTile;
    if (nblocks == 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(int64_t), st);
        return;
    }
    k_scan_reduce<<<(unsigned)nblocks, kScanThreads, 0, st>>>(in, max_count, count_ptr, capacity, partials);
    k_scan_top<<<1, 1024, 0, st>>>(partials, nblocks, total, max_count, count_ptr, capacity);
    k_scan_apply<<<(unsigned)nblocks, kScanThreads, 0, st>>>(in, out, max_count, count_ptr, capacity, partials);
}

// ---------------------------------------------------------------------------------
// Stable LSD radix sort pass (8-bit digit) of (key, value) pairs.
// ---------------------------------------------------------------------------------

// Keys [i, i + 8) as 32-bit values: two 16-byte loads of 32-bit keys or one of 16-bit keys.
__device__ __forceinline__ void ld8_keys(const uint32_t* p, int64_t i, uint32_t (&u)[8]) { ld8_u32(p, i, u); }
__device__ __forceinline__ void ld8_keys(const uint16_t* p, int64_t i, uint32_t (&u)[8]) {
    const uint4 a = *reinterpret_cast<const uint4*>(p + i);
    const uint32_t w[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int e = 0; e < 4; e++) {
        u[2 * e] = w[e] & 0xffffu;
        u[2 * e + 1] = w[e] >> 16;
    }
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const K* __restrict__ keys,
                                                             const int64_t* count_ptr, int64_t max_count,
                                                             int64_t capacity, int shift, uint32_t* hist,
                                                             int64_t nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t count = eff_count(count_ptr, max_count, capacity);
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    const int64_t mine = base + (int64_t)threadIdx.x * kSortItems;   // this thread's 8 consecutive keys
    if (mine + kSortItems <= count && aligned16(keys)) {
        uint32_t u[8];
        ld8_keys(keys, mine, u);
#pragma unroll
        for (int k = 0; k < kSortItems; k++) atomicAdd(&h[(u[k] >> shift) & 255u], 1u);
    } else {
#pragma unroll
        for (int k = 0; k < kSortItems; k++)
            if (mine + k < count) atomicAdd(&h[((uint32_t)keys[mine + k] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

struct HistIn {
    static constexpr bool kVec = true;
    const uint32_t* h;
    bool vec;
    __device__ int64_t operator()(int64_t i) const { return h[i]; }
    __device__ void load8(int64_t i, int64_t (&v)[8]) const {
        uint32_t u[8];
        ld8_u32(h, i, u);
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = u[k];
    }
};
struct HistOut {
    static constexpr bool kVec = true;
    uint32_t* h;
    bool vec;
    __device__ void operator()(int64_t i, int64_t prefix, int64_t) const { h[i] = (uint32_t)prefix; }
    __device__ void store8(int64_t i, const int64_t (&pre)[8]) const {
        uint4* q = reinterpret_cast<uint4*>(h + i);
        q[0] = make_uint4((uint32_t)pre[0], (uint32_t)pre[1], (uint32_t)pre[2], (uint32_t)pre[3]);
        q[1] = make_uint4((uint32_t)pre[4], (uint32_t)pre[5], (uint32_t)pre[6], (uint32_t)pre[7]);
    }
};

// Lanes of the warp holding the same BITS-bit value (an 8-bit digit, or with 9 bits also
// 256 for no key): one ballot per bit, keeping the lanes that agree with this lane on
// every bit.
template <int BITS>
__device__ __forceinline__ uint32_t warp_peers(uint32_t d) {
    uint32_t m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < BITS; b++) {
        const bool bit = (d >> b) & 1u;
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bal : ~bal;
    }
    return m;
}

// Each warp ranks 256 consecutive keys in order (32 at a time, warp_peers groups equal
// digits); warps' digit counts are then scanned in warp order, so the block's
// ranking -- and with the digit-major global scan, the whole pass -- is stable.  The
// block first writes its keys in sorted order to shared memory and then copies each
// digit's run to its global position, so consecutive threads write consecutive
// addresses.  Indices inside the block are 32-bit; a full block ranks 8-bit digits
// (eight ballots), the last, partial block also marks the slots without a key.
template <bool FULL, typename K>
__device__ __forceinline__ void radix_rank_block(const K* __restrict__ kb, const uint32_t* __restrict__ vb,
                                                 K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                 int nvalid, int64_t count, int shift,
                                                 const uint32_t* __restrict__ hist_scan,
                                                 int64_t nblocks, uint32_t (*wh)[256], uint32_t* bd, uint32_t* sk,
                                                 uint32_t* sv, int64_t* scan_sm) {
    constexpr int kWarps = kSortThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wbase = warp * (kSortItems * 32);
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t kk[kSortItems], vv[kSortItems], rr[kSortItems];
    // all loads first, so that they are in flight together (the ranking below orders
    // shared-memory accesses with warp barriers, which loads cannot be moved across)
#pragma unroll
    for (int it = 0; it < kSortItems; it++) {
        const int l = wbase + it * 32 + lane;
        const bool valid = FULL || l < nvalid;
        kk[it] = valid ? (uint32_t)kb[l] : 0u;
        vv[it] = valid ? vb[l] : 0u;
    }
#pragma unroll
    for (int it = 0; it < kSortItems; it++) {
        const int l = wbase + it * 32 + lane;
        const bool valid = FULL || l < nvalid;
        const uint32_t d = valid ? ((kk[it] >> shift) & 255u) : 256u;
        const uint32_t peers = FULL ? warp_peers<8>(d) : warp_peers<9>(d);
        const uint32_t cnt = valid ? wh[warp][d] : 0u;
        rr[it] = cnt + __popc(peers & lt);
        __syncwarp();
        if (valid && lane == 31 - __clz(peers)) wh[warp][d] = cnt + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    uint32_t total;
    {
        const int d = threadIdx.x;  // 256 threads, one per digit
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; w++) {
            const uint32_t c = wh[w][d];
            wh[w][d] = run;
            run += c;
        }
        total = run;
        bd[d] = hist_scan[(int64_t)d * nblocks + blockIdx.x];
    }
    // ds: start of this digit's run within the block
    const uint32_t ds = (uint32_t)block_exclusive_scan((int64_t)total, nullptr, scan_sm);
    bd[threadIdx.x] -= ds;   // global position of a block-local sorted index i of this digit: bd[d] + i
#pragma unroll
    for (int w = 0; w < kWarps; w++) wh[w][threadIdx.x] += ds;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; it++) {
        const int l = wbase + it * 32 + lane;
        if (FULL || l < nvalid) {
            const uint32_t lp = wh[warp][(kk[it] >> shift) & 255u] + rr[it];
            sk[lp] = kk[it];
            sv[lp] = vv[it];
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; it++) {
        const int i = it * kSortThreads + threadIdx.x;
        if (FULL || i < nvalid) {
            const uint32_t key = sk[i];
            const uint32_t pos = bd[(key >> shift) & 255u] + (uint32_t)i;
            if (SPLAT_OUT_OF_BOUNDS((int64_t)pos < count, kSiteScatter)) continue;
            kout[pos] = (K)key;
            vout[pos] = sv[i];
        }
    }
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const K* __restrict__ kin,
                                                                const uint32_t* __restrict__ vin,
                                                                K* __restrict__ kout,
                                                                uint32_t* __restrict__ vout,
                                                                const int64_t* count_ptr, int64_t max_count,
                                                                int64_t capacity, int shift,
                                                                const uint32_t* __restrict__ hist_scan,
                                                                int64_t nblocks) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ uint32_t wh[kWarps][256];
    __shared__ uint32_t bd[256];      // global start of each digit's run for this block, less its block start
    __shared__ uint32_t sk[kSortTile];
    __shared__ uint32_t sv[kSortTile];
    __shared__ int64_t scan_sm[9];
    for (int k = threadIdx.x; k < kWarps * 256; k += kSortThreads) (&wh[0][0])[k] = 0;
    const int64_t count = eff_count(count_ptr, max_count, capacity);
    const int64_t block0 = (int64_t)blockIdx.x * kSortTile;
    if (block0 >= count) return;  // whole block empty (uniform)
    const int nvalid = (int)min((int64_t)kSortTile, count - block0);
    __syncthreads();
    if (nvalid == kSortTile)
        radix_rank_block<true, K>(kin + block0, vin + block0, kout, vout, nvalid, count, shift, hist_scan, nblocks, wh, bd,
                               sk, sv, scan_sm);
    else
        radix_rank_block<false, K>(kin + block0, vin + block0, kout, vout, nvalid, count, shift, hist_scan, nblocks, wh,
                                bd, sk, sv, scan_sm);
}

// Sorts by bits [0, 8*passes) of the keys (32-bit, or 16-bit for at most two passes).
// Buffers ping-pong: pass p reads buffer p % 2 and writes buffer (p + 1) % 2; the result is
// in buffer passes % 2.
template <typename K>
void radix_sort(K* keys[2], uint32_t* vals[2], int passes, int64_t max_count, const int64_t* count_ptr,
                int64_t capacity, uint32_t* hist, int64_t* partials, cudaStream_t st, bool first_hist_done = false) {
    const int64_t nblocks = (max_count + kSortTile - 1) / kSortTile;
    if (nblocks == 0) return;
    for (int p = 0; p < passes; p++) {
        const int a = p & 1, b = a ^ 1;
        if (p > 0 || !first_hist_done)
            k_radix_hist<K><<<(unsigned)nblocks, kSortThreads, 0, st>>>(keys[a], count_ptr, max_count, capacity, 8 * p,
                                                                    hist, nblocks);
        device_scan(HistIn{hist, aligned16(hist)}, HistOut{hist, aligned16(hist)}, 256 * nblocks, nullptr, INT64_MAX,
                    partials, nullptr, st);
        k_radix_scatter<K><<<(unsigned)nblocks, kSortThreads, 0, st>>>(keys[a], vals[a], keys[b], vals[b], count_ptr,
                                                                   max_count, capacity, 8 * p, hist, nblocks);
    }
}

// ---------------------------------------------------------------------------------
// Frame-level binning
// ---------------------------------------------------------------------------------

struct VisIn {
    static constexpr bool kVec = true;
    const int32_t* n_tiles;
    bool vec;
    __device__ int64_t operator()(int64_t p) const { return n_tiles[p] > 0 ? 1 : 0; }
    __device__ void load8(int64_t i, int64_t (&v)[8]) const {
        uint32_t u[8];
        ld8_u32(n_tiles, i, u);
#pragma unroll
        for (int k = 0; k < 8; k++) v[k] = (int32_t)u[k] > 0 ? 1 : 0;
    }
};
struct VisOut {  // compact visible pairs with their depth bits as keys
    static constexpr bool kVec = false;
    const float4* rec;
    int64_t n;
    uint32_t* keys;
    uint32_t* vals;
    __device__ void operator()(int64_t p, int64_t prefix, int64_t v) const {
        if (!v) return;
        const int64_t s = p / n, i = p - s * n;
        const float depth = rec[rec_index((int)s, 2, n, i)].x;
        keys[prefix] = __float_as_uint(depth);
        vals[prefix] = (uint32_t)p;
    }
};

// ---------------------------------------------------------------------------------
// Emission through row items.  Every visible pair's tile box is cut into its tile rows, in
// depth order; a row item holds the pair's Gaussian, the row's first listed tile and its
// tile count -- the box's columns, or for a camera with the tile cull (support flag 4) the
// kept ones (cull_row_cols).  One scan gives every row item with tiles its first output
// slot and a compacted index; the emission maps each slot to its row item with one search.
// Work per row item and per slot is fixed whatever the size and shape of the Gaussians.
// ---------------------------------------------------------------------------------
constexpr int kEmitThreads = 256;
constexpr int kEmitItems = 8;
constexpr int kEmitTile = kEmitThreads * kEmitItems;  // output slots (or row items) per block
static_assert(kEmitTile == kSortTile, "emit blocks must be the first radix pass's blocks");
static_assert(kEmitThreads == 256, "one thread per digit of the emitted histogram");

struct RowsIn {   // tile rows of the j-th visible pair's box (depth order)
    static constexpr bool kVec = false;
    const uint32_t* sorted_pairs;
    const short4* rect;
    __device__ int64_t operator()(int64_t j) const {
        const short4 rc = rect[sorted_pairs[j]];
        return rc.w > rc.y ? (int64_t)(rc.w - rc.y) : 0;
    }
};

// Exclusive prefix of the counts.  It also records, for every 2048-item block, the owner
// whose range [prefix, prefix + count) holds the block's first item, so that no block has
// to search for it.
struct OffsetOut {
    static constexpr bool kVec = false;
    int64_t* offsets;
    uint32_t* first_owner;
    int64_t nblocks;
    __device__ void operator()(int64_t j, int64_t prefix, int64_t v) const {
        offsets[j] = prefix;
        for (int64_t b = (prefix + kEmitTile - 1) / kEmitTile; b < nblocks && b * kEmitTile < prefix + v; b++)
            first_owner[b] = (uint32_t)j;
    }
};

// Sensor s = floor(p / n) of a (sensor, Gaussian) pair index: a float estimate within one
// of the quotient, corrected.
__device__ __forceinline__ int pair_sensor(uint32_t p, int64_t n, float inv_n) {
    int s = (int)((float)p * inv_n);
    if ((uint64_t)s * (uint64_t)n > p) s--;
    else if ((uint64_t)(s + 1) * (uint64_t)n <= p) s++;
    return s;
}

// Row items [b * 2048, (b + 1) * 2048): the block stages its owners (visible pairs) and
// every thread fills the items of its slots, strided for coalesced writes.
__global__ void __launch_bounds__(kEmitThreads) k_rows(const uint32_t* __restrict__ sorted_pairs,
                                                      const int64_t* __restrict__ row_off,
                                                      const uint32_t* __restrict__ row_owner,
                                                      const int64_t* vis_count, const int64_t* n_rows,
                                                      int64_t capacity, const short4* __restrict__ rect,
                                                      const float4* __restrict__ rec, int64_t n, float inv_n,
                                                      const __grid_constant__ Frame fr, BinWorkspace w) {
    __shared__ int s_off[kEmitTile];
    __shared__ uint32_t s_p[kEmitTile];
    const int64_t total = *n_rows;
    if (total > capacity) return;   // over capacity: write nothing
    const int64_t r0 = (int64_t)blockIdx.x * kEmitTile;
    if (r0 >= total) return;
    const int64_t V = *vis_count;
    const int nr = (int)min((int64_t)kEmitTile, total - r0);
    const int64_t jlo = row_owner[blockIdx.x];
    const int64_t jhi = r0 + kEmitTile < total ? (int64_t)row_owner[blockIdx.x + 1] + 1 : V;
    const int nown = (int)min((int64_t)kEmitTile, jhi - jlo);
    for (int q = threadIdx.x; q < nown; q += kEmitThreads) {
        s_off[q] = (int)(row_off[jlo + q] - r0);
        s_p[q] = sorted_pairs[jlo + q];
    }
    __syncthreads();
#pragma unroll 2
    for (int it = 0; it < kEmitItems; it++) {
        const int r = it * kEmitThreads + threadIdx.x;
        if (r >= nr) break;
        int lo = 0, hi = nown - 1;   // last owner with s_off <= r
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= r) lo = mid;
            else hi = mid - 1;
        }
        const uint32_t p = s_p[lo];
        const int s = pair_sensor(p, n, inv_n);
        const uint32_t id = (uint32_t)(p - (uint64_t)s * (uint64_t)n);
        const short4 rc = rect[p];
        const SensorDev& S = fr.s[s];
        const int tx = S.tiles_x, wd = rc.z - rc.x, row = rc.y + (r - s_off[lo]);
        const bool ok = rc.x >= 0 && rc.x < tx && wd > 0 && wd <= tx && rc.y >= 0 && rc.w > rc.y &&
                        rc.w <= S.tiles_y;   // else a malformed projection: listed nowhere
        int ca = rc.x, cnt = ok ? wd : 0;
        if (ok && S.kind == SPLAT_SENSOR_CAMERA && (S.support & 4)) {
            const float4 g0 = rec[rec_index(s, 0, n, id)], g1 = rec[rec_index(s, 1, n, id)];
            const CullGauss cg = cull_setup(g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w);
            int cb;
            cull_row_cols(S, cg, row, rc.x, rc.z, &ca, &cb);
            cnt = cb - ca;
        }
        const int64_t j = r0 + r;
        w.r_key0[j] = (uint32_t)(S.tile_base + row * tx + ca);
        w.r_id[j] = id;
        w.r_wrap[j] = S.kind == SPLAT_SENSOR_LIDAR ? tx - ca : 0x7fffffff;   // lidar azimuth wrap
        w.r_tx[j] = tx;
        w.r_cnt[j] = cnt;
    }
}

// Slots and compaction in one scan: the low 32 bits count a row item's tiles, the high 32
// bits whether it has any (the sums stay below 2^31 each, so no carry crosses).
struct SlotIn {
    static constexpr bool kVec = true;
    const int32_t* cnt;
    bool vec;
    __device__ int64_t operator()(int64_t j) const {
        const int64_t c = cnt[j];
        return c | ((int64_t)(c > 0) << 32);
    }
    __device__ void load8(int64_t i, int64_t (&v)[8]) const {
        uint32_t u[8];
        ld8_u32(cnt, i, u);
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const int64_t c = (int32_t)u[k];
            v[k] = c | ((int64_t)(c > 0) << 32);
        }
    }
};
struct SlotOut {
    static constexpr bool kVec = false;
    int32_t* c_off;
    int32_t* c_row;
    uint32_t* first_owner;
    int64_t nblocks;
    __device__ void operator()(int64_t j, int64_t prefix, int64_t v) const {
        const int64_t c = v & 0xffffffff;
        if (c <= 0) return;
        const int64_t slot = prefix & 0xffffffff, k = prefix >> 32;
        c_off[k] = (int32_t)slot;
        c_row[k] = (int32_t)j;
        for (int64_t b = (slot + kEmitTile - 1) / kEmitTile; b < nblocks && b * kEmitTile < slot + c; b++)
            first_owner[b] = (uint32_t)k;
    }
};

// The totals: intersections (or, when the row items overflowed the capacity, the capacity
// needed) and the row items with tiles.
__global__ void k_slot_totals(const int64_t* n_rows, int64_t capacity, const int64_t* slot_total, int64_t* n_isect,
                              int64_t* n_owners) {
    const int64_t r = *n_rows;
    if (r > capacity) {
        *n_isect = r;
        *n_owners = 0;
    } else {
        *n_isect = *slot_total & 0xffffffff;
        *n_owners = *slot_total >> 32;
    }
}

// Writes intersections [b*2048, (b+1)*2048): the slot scan recorded the row item that owns
// each block's first slot; the block stages its owners (first slot, first tile, Gaussian,
// wrap) in shared memory and every thread writes the consecutive slots [8 t, 8 t + 8): one
// search for the owner of the first, then each slot's tile is the owner's first tile plus
// its offset (less a lidar row's column count past its wrap).  The writes are contiguous.
// The blocks are those of the first radix pass over the keys, so each block also writes
// that pass's low-byte digit histogram.  Keys are 16-bit when every tile id fits.
template <typename Key>
__global__ void __launch_bounds__(kEmitThreads) k_emit(const BinWorkspace w, const int64_t* n_isect,
                                                      int64_t capacity, Key* __restrict__ keys,
                                                      uint32_t* __restrict__ vals, uint32_t* __restrict__ hist) {
    __shared__ int s_off[kEmitTile];
    __shared__ uint32_t s_key0[kEmitTile];
    __shared__ uint32_t s_id[kEmitTile];
    __shared__ int s_wrap[kEmitTile];
    __shared__ int s_tx[kEmitTile];
    __shared__ uint32_t s_hist[256];   // low-byte digit counts of this block's keys (first radix pass)
    const int64_t total = *n_isect;
    if (total > capacity) return;   // over capacity: write nothing
    const int64_t o0 = (int64_t)blockIdx.x * kEmitTile;
    const int64_t nblocks = gridDim.x;   // the radix passes cut the keys into the same 2048-slot blocks
    if (o0 >= total) {
        hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = 0;
        return;
    }
    s_hist[threadIdx.x] = 0;
    const int64_t K = *w.n_owners;
    const int nslot = (int)min((int64_t)kEmitTile, total - o0);
    if (SPLAT_OUT_OF_BOUNDS(o0 + nslot <= capacity, kSiteEmit)) return;
    const int64_t jlo = w.first_owner[blockIdx.x];
    // owners of this block's slots are jlo .. the owner of the next block's first slot (at
    // most kEmitTile of them with a slot here: every compacted row item owns a slot)
    const int64_t jhi = o0 + kEmitTile < total ? (int64_t)w.first_owner[blockIdx.x + 1] + 1 : K;
    const int nown = (int)min((int64_t)kEmitTile, jhi - jlo);
    for (int q = threadIdx.x; q < nown; q += kEmitThreads) {
        const int64_t k = jlo + q;
        const int r = w.c_row[k];
        s_off[q] = (int)(w.c_off[k] - o0);
        s_key0[q] = w.r_key0[r];
        s_id[q] = w.r_id[r];
        s_wrap[q] = w.r_wrap[r];
        s_tx[q] = w.r_tx[r];
    }
    __syncthreads();
    const int ofirst = kEmitItems * threadIdx.x;
    if (ofirst < nslot) {
        int cur = 0, hi = nown - 1;   // last owner with s_off <= ofirst
        while (cur < hi) {
            const int mid = (cur + hi + 1) >> 1;
            if (s_off[mid] <= ofirst) cur = mid;
            else hi = mid - 1;
        }
        int next = cur + 1 < nown ? s_off[cur + 1] : kEmitTile;
        uint32_t kk[kEmitItems], vv[kEmitItems];
#pragma unroll
        for (int i = 0; i < kEmitItems; i++) {
            const int o = ofirst + i;
            if (o >= next) {   // every owner holds at least one slot: the walk enters the next at its start
                cur++;
                next = cur + 1 < nown ? s_off[cur + 1] : kEmitTile;
            }
            const int dx = o - s_off[cur];
            const uint32_t key = s_key0[cur] + (uint32_t)dx - (dx >= s_wrap[cur] ? (uint32_t)s_tx[cur] : 0u);
            kk[i] = key;
            vv[i] = s_id[cur];
            if (o < nslot) atomicAdd(&s_hist[key & 255u], 1u);
        }
        // vector stores when both arrays are 16-byte aligned (the workspace always is; the
        // caller's list may be the value array)
        const bool vec = ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(vals)) & 15u) == 0;
        if (vec && ofirst + kEmitItems <= nslot) {
            uint4* kp = reinterpret_cast<uint4*>(keys + o0 + ofirst);
            uint4* vp = reinterpret_cast<uint4*>(vals + o0 + ofirst);
            if constexpr (sizeof(Key) == 2) {
                kp[0] = make_uint4(kk[0] | (kk[1] << 16), kk[2] | (kk[3] << 16), kk[4] | (kk[5] << 16),
                                   kk[6] | (kk[7] << 16));
            } else {
                kp[0] = make_uint4(kk[0], kk[1], kk[2], kk[3]);
                kp[1] = make_uint4(kk[4], kk[5], kk[6], kk[7]);
            }
            vp[0] = make_uint4(vv[0], vv[1], vv[2], vv[3]);
            vp[1] = make_uint4(vv[4], vv[5], vv[6], vv[7]);
        } else {
#pragma unroll
            for (int i = 0; i < kEmitItems; i++) {
                if (ofirst + i < nslot) {
                    keys[o0 + ofirst + i] = (Key)kk[i];
                    vals[o0 + ofirst + i] = vv[i];
                }
            }
        }
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = s_hist[threadIdx.x];
}

// Tile ranges of the sorted ids: four keys per thread (one vector load) plus the two
// neighbours; keys past every tile (malformed projections) are never ranged.
__device__ __forceinline__ void ld4_keys(const uint32_t* p, int64_t j, uint32_t* k) {
    const uint4 v = *reinterpret_cast<const uint4*>(p + j);
    k[0] = v.x;
    k[1] = v.y;
    k[2] = v.z;
    k[3] = v.w;
}
__device__ __forceinline__ void ld4_keys(const uint16_t* p, int64_t j, uint32_t* k) {
    const uint2 v = *reinterpret_cast<const uint2*>(p + j);
    k[0] = v.x & 0xffffu;
    k[1] = v.x >> 16;
    k[2] = v.y & 0xffffu;
    k[3] = v.y >> 16;
}

template <typename K>
__global__ void __launch_bounds__(256) k_tile_ranges(const K* __restrict__ keys, const int64_t* count_ptr,
                                                      int64_t capacity, int64_t total_tiles, int2* ranges) {
    const int64_t count = eff_count(count_ptr, capacity, capacity);
    const int64_t groups = (count + 3) / 4;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < groups;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j0 = 4 * q;
        uint32_t k[6];   // k[1 + i] = keys[j0 + i]; k[0], k[5]: neighbours
        if (j0 + 4 <= count) {
            ld4_keys(keys, j0, k + 1);
        } else {
#pragma unroll
            for (int i = 0; i < 4; i++) k[1 + i] = j0 + i < count ? (uint32_t)keys[j0 + i] : 0u;
        }
        k[0] = j0 > 0 ? (uint32_t)keys[j0 - 1] : 0u;
        k[5] = j0 + 4 < count ? (uint32_t)keys[j0 + 4] : 0u;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int64_t j = j0 + i;
            if (j >= count) break;
            const uint32_t t = k[1 + i];
            if ((int64_t)t >= total_tiles) continue;
            if (j == 0 || k[i] != t) ranges[t].x = (int)j;
            if (j == count - 1 || k[2 + i] != t) ranges[t].y = (int)(j + 1);
        }
    }
}

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace carving; with base == nullptr only computes the size.
BinWorkspace carve_workspace(void* base, int64_t pairs, int64_t capacity) {
    BinWorkspace w{};
    char* p = (char*)base;
    size_t off = 0;
    auto take = [&](size_t bytes) -> void* {
        void* r = p ? (void*)(p + off) : nullptr;
        off += align_up(bytes);
        return r;
    };
    const int64_t vp = pairs > 0 ? pairs : 1, cp = capacity > 0 ? capacity : 1;
    w.vkeys[0] = (uint32_t*)take(4 * vp);
    w.vkeys[1] = (uint32_t*)take(4 * vp);
    w.vvals[0] = (uint32_t*)take(4 * vp);
    w.vvals[1] = (uint32_t*)take(4 * vp);
    w.vis_count = (int64_t*)take(8);
    w.offsets = (int64_t*)take(8 * vp);
    w.row_owner = (uint32_t*)take(4 * ((cp + kEmitTile - 1) / kEmitTile + 1));
    w.n_rows = (int64_t*)take(8);
    w.r_key0 = (uint32_t*)take(4 * cp);
    w.r_id = (uint32_t*)take(4 * cp);
    w.r_wrap = (int32_t*)take(4 * cp);
    w.r_tx = (int32_t*)take(4 * cp);
    w.r_cnt = (int32_t*)take(4 * cp);
    w.c_off = (int32_t*)take(4 * cp);
    w.c_row = (int32_t*)take(4 * cp);
    w.slot_total = (int64_t*)take(8);
    w.n_owners = (int64_t*)take(8);
    w.ikeys[0] = (uint32_t*)take(4 * cp);
    w.ikeys[1] = (uint32_t*)take(4 * cp);
    w.ivals_tmp = (uint32_t*)take(4 * cp);
    w.first_owner = (uint32_t*)take(4 * ((cp + kEmitTile - 1) / kEmitTile));
    const int64_t maxn = vp > cp ? vp : cp;
    const int64_t sort_blocks = (maxn + kSortTile - 1) / kSortTile;
    w.hist = (uint32_t*)take(4 * 256 * sort_blocks);
    const int64_t scan_items = (256 * sort_blocks > maxn ? 256 * sort_blocks : maxn);
    w.partials = (int64_t*)take(8 * ((scan_items + kScanTile - 1) / kScanTile + 1));
    w.bytes = off;
    return w;
}

static int bits_for(int64_t v) {
    int b = 0;
    while (b < 62 && ((int64_t)1 << b) < v) b++;
    return b;
}

template <typename K>
static void tile_stage(const BinWorkspace& w, K* keys[2], uint32_t* vals_buf[2], int passes, int64_t capacity,
                       int64_t emit_blocks, int64_t* n_isect, int64_t total_tiles, int2* tile_ranges,
                       cudaStream_t st) {
    if (emit_blocks > 0)
        k_emit<K><<<(unsigned)emit_blocks, kEmitThreads, 0, st>>>(w, n_isect, capacity, keys[0], vals_buf[0], w.hist);
    radix_sort<K>(keys, vals_buf, passes, capacity, n_isect, capacity, w.hist, w.partials, st, emit_blocks > 0);
    int64_t blocks = (capacity + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks > 0)
        k_tile_ranges<K><<<(unsigned)blocks, 256, 0, st>>>(keys[passes & 1], n_isect, capacity, total_tiles,
                                                           tile_ranges);
}

void launch_bin_sort(const Frame& fr, int64_t n, const float4* rec, const short4* rect, const int32_t* n_tiles,
                     int64_t capacity, uint32_t* isect_ids, int2* tile_ranges, int64_t total_tiles,
                     int64_t* n_isect, void* workspace, cudaStream_t st) {
    BinWorkspace w = carve_workspace(workspace, (int64_t)fr.n_sensors * n, capacity);
    const int64_t pairs = (int64_t)fr.n_sensors * n;
    cudaMemsetAsync(tile_ranges, 0, sizeof(int2) * (size_t)total_tiles, st);
    // 1. compact visible pairs (stable), keyed by depth bits
    device_scan(VisIn{n_tiles, aligned16(n_tiles)}, VisOut{rec, n, w.vkeys[0], w.vvals[0]}, pairs, nullptr, INT64_MAX, w.partials,
                w.vis_count, st);
    // 2. stable depth sort of the visible pairs (32-bit keys)
    radix_sort<uint32_t>(w.vkeys, w.vvals, 4, pairs, w.vis_count, INT64_MAX, w.hist, w.partials, st);
    const uint32_t* sorted_pairs = w.vvals[0];  // 4 passes: result back in buffer 0
    // 3. emit (tile, id) in depth order; n_isect = total
    const int passes = (bits_for(total_tiles) + 7) / 8 > 0 ? (bits_for(total_tiles) + 7) / 8 : 1;
    uint32_t* vals_buf[2];
    // the result lands in buffer passes % 2: make that buffer the caller's isect_ids
    vals_buf[passes & 1] = isect_ids;
    vals_buf[(passes & 1) ^ 1] = w.ivals_tmp;
    const int64_t emit_blocks = (capacity + kEmitTile - 1) / kEmitTile;
    // 3a. row items: the tile rows of the visible pairs' boxes, in depth order
    device_scan(RowsIn{sorted_pairs, rect}, OffsetOut{w.offsets, w.row_owner, emit_blocks}, pairs, w.vis_count,
                INT64_MAX, w.partials, w.n_rows, st);
    if (emit_blocks > 0)
        k_rows<<<(unsigned)emit_blocks, kEmitThreads, 0, st>>>(sorted_pairs, w.offsets, w.row_owner, w.vis_count,
                                                               w.n_rows, capacity, rect, rec, n,
                                                               (float)(1.0 / (double)n), fr, w);
    // 3b. each row item's first slot, the row items with tiles compacted; n_isect = total
    device_scan(SlotIn{w.r_cnt, aligned16(w.r_cnt)}, SlotOut{w.c_off, w.c_row, w.first_owner, emit_blocks}, capacity, w.n_rows, capacity,
                w.partials, w.slot_total, st);
    k_slot_totals<<<1, 1, 0, st>>>(w.n_rows, capacity, w.slot_total, n_isect, w.n_owners);
    // 3c.-5. the intersections, their stable sort by tile id and the per-tile ranges, with
    // 16-bit keys when every tile id fits (the key buffers hold 32 bits per slot either way)
    if (total_tiles <= 65536) {
        uint16_t* k16[2] = {reinterpret_cast<uint16_t*>(w.ikeys[0]), reinterpret_cast<uint16_t*>(w.ikeys[1])};
        tile_stage(w, k16, vals_buf, passes, capacity, emit_blocks, n_isect, total_tiles, tile_ranges, st);
    } else {
        tile_stage(w, w.ikeys, vals_buf, passes, capacity, emit_blocks, n_isect, total_tiles, tile_ranges, st);
    }
}

}  // namespace splat
