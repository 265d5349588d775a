// rays.cu -- lidar point clouds as rays (App. A.2) and their grouping by tile.
//
// A captured point is stored in the sensor frame of the sweep's reference time (ego
// motion compensated).  Rendering it needs the ray it was measured along: the
// compensation is removed with the sensor's constant linear and angular velocity (the
// motion model of the rolling-shutter projection), q = p - t (v + omega x p), and the ray
// is q's azimuth, elevation and the capture time.  Each ray belongs to the tile of a
// zero-extent Gaussian at its (azimuth, elevation): column floor(phi / w_phi), the row
// whose elevation boundaries hold omega, none outside the beam fan.
//
// The grouping is a counting sort by tile: count (atomics into the range table), one
// block scans the counts into tile starts and 256-ray chunk numbers, scatter (atomic
// cursors).  The order of the rays inside a tile is unspecified; every ray is rendered on
// its own, so the outputs do not depend on it.
#include "status.cuh"
#include "types.cuh"

namespace splat {

constexpr int kRayThreads = 256;
constexpr int kScanThreads = 1024;

// Tile of a free ray within its lidar (-1: outside the beam fan).
__device__ __forceinline__ int free_ray_tile(const SensorDev& S, float phi, float om) {
    const int Mw = S.nb / S.tile_h;
    if (!(om > elev_bound(S, 0)) || !(om < elev_bound(S, Mw)) || !(phi >= 0.f) || !(phi < kTwoPi)) return -1;
    const int c = min((int)floorf(phi / S.wphi), S.tiles_x - 1);
    int row = 0;
    for (int k = 1; k < Mw; k++)
        if (elev_bound(S, k) <= om) row = k;
    return row * S.tiles_x + c;
}

__global__ void __launch_bounds__(kRayThreads)
    k_points_to_rays(const SensorDev S, const float* __restrict__ pts, const float* __restrict__ times, int64_t n,
                     float* __restrict__ rays, float* __restrict__ range, int32_t* __restrict__ tiles) {
    const int64_t i = (int64_t)blockIdx.x * kRayThreads + threadIdx.x;
    if (i >= n) return;
    const float px = pts[3 * i], py = pts[3 * i + 1], pz = pts[3 * i + 2];
    const float t = times[i];
    // q = p - t (v + omega x p): the point in the sensor frame of its capture time
    const float cx = S.w[1] * pz - S.w[2] * py;
    const float cy = S.w[2] * px - S.w[0] * pz;
    const float cz = S.w[0] * py - S.w[1] * px;
    const float qx = px - t * (S.v[0] + cx);
    const float qy = py - t * (S.v[1] + cy);
    const float qz = pz - t * (S.v[2] + cz);
    const float r = sqrtf(qx * qx + qy * qy + qz * qz);
    float phi = atan2f(qy, qx);
    if (phi < 0.f) phi += kTwoPi;
    if (phi >= kTwoPi) phi -= kTwoPi;   // a tiny negative angle rounds up to 2 pi
    const float om = asinf(fminf(fmaxf(qz / fmaxf(r, 1e-30f), -1.f), 1.f));
    rays[3 * i] = phi;
    rays[3 * i + 1] = om;
    rays[3 * i + 2] = t;
    range[i] = r;
    if (tiles) tiles[i] = free_ray_tile(S, phi, om);
}

__global__ void __launch_bounds__(kRayThreads)
    k_ray_count(const SensorDev S, const float* __restrict__ rays, int64_t n, int2* __restrict__ ranges) {
    const int64_t i = (int64_t)blockIdx.x * kRayThreads + threadIdx.x;
    if (i >= n) return;
    const int tile = free_ray_tile(S, rays[3 * i], rays[3 * i + 1]);
    if (SPLAT_OUT_OF_BOUNDS(tile < S.tiles_x * S.tiles_y, kSiteRayTile)) return;
    if (tile >= 0) atomicAdd(&ranges[tile].y, 1);
}

// Exclusive prefix over the block of two per-thread values (threads in order); also the
// block totals.  Every thread of the kScanThreads-thread block calls it.
__device__ __forceinline__ void block_scan2(int& a, int& b, int& tot_a, int& tot_b) {
    __shared__ int s_a[kScanThreads / 32], s_b[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, ia, o), y = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += x;
            ib += y;
        }
    }
    if (lane == 31) {
        s_a[warp] = ia;
        s_b[warp] = ib;
    }
    __syncthreads();
    if (warp == 0) {
        int x = s_a[lane], y = s_b[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, x, o), v = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) {
                x += u;
                y += v;
            }
        }
        s_a[lane] = x;   // inclusive totals of warps 0..lane
        s_b[lane] = y;
    }
    __syncthreads();
    a = ia - a + (warp > 0 ? s_a[warp - 1] : 0);
    b = ib - b + (warp > 0 ? s_b[warp - 1] : 0);
    tot_a = s_a[kScanThreads / 32 - 1];
    tot_b = s_b[kScanThreads / 32 - 1];
}

// One block over the tiles, each thread a contiguous run of them.  Counts are taken from
// src (end - start, at most cap) or, without src, from .y of dst (the count kernel's
// atomics).  dst[t] becomes (start, start) -- the scatter cursor -- or, with src,
// (start, start + count); chunk_base[t] the first 256-ray chunk of the tile.
__global__ void __launch_bounds__(kScanThreads) k_ray_scan(const int2* __restrict__ src, int2* __restrict__ dst,
                                                           int tiles, int cap, int32_t* __restrict__ chunk_base) {
    const int per = (tiles + kScanThreads - 1) / kScanThreads;
    const int t0 = min(tiles, (int)threadIdx.x * per), t1 = min(tiles, t0 + per);
    auto count = [&](int t) { return src ? min(src[t].y - src[t].x, cap) : dst[t].y; };
    int cnt = 0, chk = 0;
    for (int t = t0; t < t1; t++) {
        const int c = count(t);
        cnt += c;
        chk += (c + kListChunk - 1) / kListChunk;
    }
    int tot_cnt, tot_chk;
    block_scan2(cnt, chk, tot_cnt, tot_chk);
    for (int t = t0; t < t1; t++) {
        const int c = count(t);
        dst[t] = make_int2(cnt, src ? cnt + c : cnt);
        chunk_base[t] = chk;
        cnt += c;
        chk += (c + kListChunk - 1) / kListChunk;
    }
    if (threadIdx.x == kScanThreads - 1) chunk_base[tiles] = tot_chk;
}

__global__ void __launch_bounds__(kRayThreads)
    k_ray_scatter(const SensorDev S, const float* __restrict__ rays, int64_t n, int2* __restrict__ ranges,
                  int32_t* __restrict__ ids) {
    const int64_t i = (int64_t)blockIdx.x * kRayThreads + threadIdx.x;
    if (i >= n) return;
    const int tile = free_ray_tile(S, rays[3 * i], rays[3 * i + 1]);
    if (SPLAT_OUT_OF_BOUNDS(tile < S.tiles_x * S.tiles_y, kSiteRayTile)) return;
    if (tile >= 0) {
        const int slot = atomicAdd(&ranges[tile].y, 1);
        if (SPLAT_OUT_OF_BOUNDS(slot >= 0 && slot < n, kSiteRaySlot)) return;
        ids[slot] = (int32_t)i;
    }
}

void launch_points_to_rays(const SensorDev& S, const float* points, const float* times, int64_t n, float* rays,
                           float* range, int32_t* tiles, cudaStream_t st) {
    if (n <= 0) return;
    const int64_t blocks = (n + kRayThreads - 1) / kRayThreads;
    k_points_to_rays<<<(unsigned)blocks, kRayThreads, 0, st>>>(S, points, times, n, rays, range, tiles);
}

void launch_bin_rays(const SensorDev& S, const float* rays, int64_t n, int32_t* ids, int2* ranges,
                     int32_t* chunk_base, cudaStream_t st) {
    const int tiles = S.tiles_x * S.tiles_y;
    cudaMemsetAsync(ranges, 0, sizeof(int2) * (size_t)tiles, st);
    const int64_t blocks = (n + kRayThreads - 1) / kRayThreads;
    if (n > 0) k_ray_count<<<(unsigned)blocks, kRayThreads, 0, st>>>(S, rays, n, ranges);
    k_ray_scan<<<1, kScanThreads, 0, st>>>(nullptr, ranges, tiles, 0, chunk_base);
    if (n > 0) k_ray_scatter<<<(unsigned)blocks, kRayThreads, 0, st>>>(S, rays, n, ranges, ids);
}

// Training-time cap (App. A.2): a tile keeps the `cap` rays of smallest (priority, ray
// index); the caller draws fresh priorities each iteration, which shuffles the rays a full
// tile keeps.  One block per tile: each ray's rank is the number of the tile's rays with a
// smaller key (keys staged through shared memory); rank < cap writes the ray to slot
// start + rank of the capped list, so the kept rays come out in key order.
constexpr int kCapStage = 1024;
__global__ void __launch_bounds__(kRayThreads)
    k_ray_cap(const int2* __restrict__ src_ranges, const int32_t* __restrict__ src_ids,
              const uint32_t* __restrict__ prio, int cap, const int2* __restrict__ dst_ranges,
              int32_t* __restrict__ dst_ids) {
    __shared__ unsigned long long s_key[kCapStage];
    const int2 sr = src_ranges[blockIdx.x];
    const int cnt = sr.y - sr.x, out0 = dst_ranges[blockIdx.x].x;
    auto key_of = [&](int id) { return ((unsigned long long)prio[id] << 32) | (uint32_t)id; };
    for (int j0 = 0; j0 < cnt; j0 += kRayThreads) {
        const int j = j0 + threadIdx.x;
        const int id = j < cnt ? src_ids[sr.x + j] : 0;
        const unsigned long long kj = key_of(id);
        int rank = 0;
        for (int k0 = 0; k0 < cnt; k0 += kCapStage) {
            const int nk = min(kCapStage, cnt - k0);
            __syncthreads();
            for (int k = threadIdx.x; k < nk; k += kRayThreads) s_key[k] = key_of(src_ids[sr.x + k0 + k]);
            __syncthreads();
            for (int k = 0; k < nk; k++) rank += s_key[k] < kj;
        }
        if (j < cnt && rank < cap) dst_ids[out0 + rank] = id;
    }
}

void launch_bin_rays_capped(const SensorDev& S, const float* rays, const uint32_t* priority, int64_t n, int cap,
                            int32_t* tmp_ids, int2* tmp_ranges, int32_t* tmp_chunks, int32_t* ids, int2* ranges,
                            int32_t* chunk_base, cudaStream_t st) {
    launch_bin_rays(S, rays, n, tmp_ids, tmp_ranges, tmp_chunks, st);
    const int tiles = S.tiles_x * S.tiles_y;
    k_ray_scan<<<1, kScanThreads, 0, st>>>(tmp_ranges, ranges, tiles, cap, chunk_base);
    if (n > 0) k_ray_cap<<<tiles, kRayThreads, 0, st>>>(tmp_ranges, tmp_ids, priority, cap, ranges, ids);
}

}  // namespace splat
