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
    if (tile >= 0) atomicAdd(&ranges[tile].y, 1);
}

// One block: counts (in .y) -> (start, start) with the cursor in .y, and chunk numbers.
// Each thread takes a contiguous run of tiles; a block-wide exclusive scan of the run
// totals gives each run its base.
__global__ void __launch_bounds__(kScanThreads) k_ray_scan(int2* __restrict__ ranges, int tiles,
                                                           int32_t* __restrict__ chunk_base) {
    __shared__ int s_cnt[kScanThreads / 32], s_chk[kScanThreads / 32];
    const int per = (tiles + kScanThreads - 1) / kScanThreads;
    const int t0 = min(tiles, (int)threadIdx.x * per), t1 = min(tiles, t0 + per);
    int cnt = 0, chk = 0;
    for (int t = t0; t < t1; t++) {
        const int c = ranges[t].y;
        cnt += c;
        chk += (c + kListChunk - 1) / kListChunk;
    }
    // inclusive warp scans, then the warp totals
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int ic = cnt, ik = chk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, ic, o), b = __shfl_up_sync(0xffffffffu, ik, o);
        if (lane >= o) {
            ic += a;
            ik += b;
        }
    }
    if (lane == 31) {
        s_cnt[warp] = ic;
        s_chk[warp] = ik;
    }
    __syncthreads();
    if (warp == 0) {
        int a = s_cnt[lane], b = s_chk[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, a, o), y = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) {
                a += x;
                b += y;
            }
        }
        s_cnt[lane] = a;   // inclusive totals of warps 0..lane
        s_chk[lane] = b;
    }
    __syncthreads();
    int base = ic - cnt + (warp > 0 ? s_cnt[warp - 1] : 0);
    int cbase = ik - chk + (warp > 0 ? s_chk[warp - 1] : 0);
    for (int t = t0; t < t1; t++) {
        const int c = ranges[t].y;
        ranges[t] = make_int2(base, base);
        chunk_base[t] = cbase;
        base += c;
        cbase += (c + kListChunk - 1) / kListChunk;
    }
    if (threadIdx.x == kScanThreads - 1) chunk_base[tiles] = s_chk[kScanThreads / 32 - 1];
}

__global__ void __launch_bounds__(kRayThreads)
    k_ray_scatter(const SensorDev S, const float* __restrict__ rays, int64_t n, int2* __restrict__ ranges,
                  int32_t* __restrict__ ids) {
    const int64_t i = (int64_t)blockIdx.x * kRayThreads + threadIdx.x;
    if (i >= n) return;
    const int tile = free_ray_tile(S, rays[3 * i], rays[3 * i + 1]);
    if (tile >= 0) ids[atomicAdd(&ranges[tile].y, 1)] = (int32_t)i;
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
    k_ray_scan<<<1, kScanThreads, 0, st>>>(ranges, tiles, chunk_base);
    if (n > 0) k_ray_scatter<<<(unsigned)blocks, kRayThreads, 0, st>>>(S, rays, n, ranges, ids);
}

}  // namespace splat
