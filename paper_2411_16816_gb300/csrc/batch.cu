// batch.cu -- one persistent launch that rasterizes many camera views and lidar sweeps of
// different sizes, over several scenes (a serving batch).
//
// The requests' projections and sorted tile lists come from the per-frame entry points
// (splat_project / splat_bin_sort on groups of sensors); this launch then renders every
// (request, tile) work item.  Blocks stay resident (one wave of CTAs) and pull items from
// an atomic counter, so large and small requests, cameras and lidars, share the machine
// without a tail of idle SMs; each request may use its own 256-ray tile shape.  The end
// of each request is stamped with the device's global timer for latency measurement.
// No block ever waits for another: the counter is only incremented.
#include <cstring>

#include "raster_impl.cuh"

namespace splat {
splat_status record_error(splat_status code, const char* msg);
splat_status frame_sensor_constants(int32_t n_sensors, const splat_sensor* sensors, int32_t which, SensorDev* out);
}

namespace splat {

constexpr int kBatchThreads = 128;   // two rays per thread: one 256-ray tile per work item
constexpr int kBatchPX = 2;
constexpr int kMaxBatch = 1024;

struct BatchReqDev {
    SensorDev S;              // ray_base = 0: every request has its own outputs
    const float4* rec;        // its group's projected records [S][3][n]
    const uint32_t* ids;      // its group's sorted lists
    const int2* ranges;       // its group's tile ranges
    const float* feat;        // its scene's features [n][C]
    int64_t n;
    int C;
    int sensor_index;         // index of the sensor in its group
    int tiles;
    int pad;
    const int64_t* n_isect;   // its group's intersection count
    int64_t item_base;        // first work item of this request
    float* out_feat;
    float* out_T;
    float* out_range_exp;
    float* out_range_med;
    float* out_alpha;
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int CM, bool LIDAR, bool COUNT>
__device__ __forceinline__ void batch_tile(const BatchReqDev& B, int lt, unsigned char* smem_raw,
                                           unsigned long long* evaluated) {
    constexpr int PX = kBatchPX;
    Stage<CM, kBatchThreads, LIDAR>& sm = *reinterpret_cast<Stage<CM, kBatchThreads, LIDAR>*>(smem_raw);
    const SensorDev& S = B.S;
    TileCtx tc;
    tc.s = B.sensor_index;
    tc.tx = lt % S.tiles_x;
    tc.ty = lt / S.tiles_x;
    tc.gtile = S.tile_base + lt;
    RayCtx r[PX];
#pragma unroll
    for (int q = 0; q < PX; q++)
        r[q] = ray_setup_rt<LIDAR>(S, tc.tx, tc.ty, threadIdx.x + q * kBatchThreads, S.tile_w, S.tile_h);
    RasterIn in{B.rec, B.ids, B.ranges, B.feat, B.n, B.C};
    in.n_isect = B.n_isect;
    const int2 range = load_range(in, tc.gtile);
    TileBox box{};
    if (!LIDAR) box = camera_tile_box(S, tc.tx, tc.ty, S.tile_w, S.tile_h);
    float2 F[PX][CM / 2];
#pragma unroll
    for (int q = 0; q < PX; q++)
#pragma unroll
        for (int c = 0; c < CM / 2; c++) F[q][c] = make_float2(0.f, 0.f);
    FwdState st[PX];
    // 16 x 16 only fixes the 256-ray batch size here; the ray layout comes from r[].
    const int evals = forward_tile<CM, 16, 16, LIDAR, PX, true, COUNT>(sm, in, tc, box, r, range, st, F);
    if (COUNT) {
        unsigned long long e = (unsigned long long)evals;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if ((threadIdx.x & 31) == 0 && e) atomicAdd(evaluated + (LIDAR ? 1 : 0), e);
    }
    const int C = B.C;
#pragma unroll
    for (int q = 0; q < PX; q++) {
        if (!r[q].inside) continue;
        const int64_t o = r[q].o;
        float* fo = B.out_feat + o * C;
        if ((C & 3) == 0) {
#pragma unroll
            for (int c = 0; c < CM; c += 4)
                if (c < C)
                    *reinterpret_cast<float4*>(fo + c) =
                        make_float4(F[q][c / 2].x, F[q][c / 2].y, F[q][c / 2 + 1].x, F[q][c / 2 + 1].y);
        } else {
#pragma unroll
            for (int c = 0; c < CM; c++)
                if (c < C) fo[c] = (c & 1) ? F[q][c / 2].y : F[q][c / 2].x;
        }
        if (B.out_T) B.out_T[o] = st[q].T;
        if (LIDAR) {
            B.out_range_exp[o] = st[q].de;
            if (B.out_range_med) B.out_range_med[o] = st[q].dm;
            B.out_alpha[o] = 1.f - st[q].T;
        }
    }
}

template <int CM, bool COUNT>
__global__ void __launch_bounds__(kBatchThreads, 4) k_raster_batch(const BatchReqDev* __restrict__ tab, int n_req,
                                                               int64_t total, int* counters,
                                                               unsigned long long* stamps,
                                                               unsigned long long* evaluated) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int64_t s_base[kMaxBatch + 1];
    __shared__ int64_t s_item;
    for (int q = threadIdx.x; q < n_req; q += kBatchThreads) s_base[q] = tab[q].item_base;
    if (threadIdx.x == 0) s_base[n_req] = total;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(&counters[n_req], 1);
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        int lo = 0, hi = n_req - 1;   // last request whose first item is <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_base[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const BatchReqDev& B = tab[lo];
        const int lt = (int)(item - s_base[lo]);
        if (B.S.kind == SPLAT_SENSOR_CAMERA) batch_tile<CM, false, COUNT>(B, lt, smem_raw, evaluated);
        else batch_tile<CM, true, COUNT>(B, lt, smem_raw, evaluated);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const int done = atomicAdd(&counters[lo], 1) + 1;
            if (stamps && done == B.tiles) stamps[lo] = global_ns();
        }
    }
}

__global__ void k_stamp(unsigned long long* at) { *at = global_ns(); }

template <int CM>
static splat_status launch_batch_t(const BatchReqDev* tab, int n_req, int64_t total, int* counters,
                                   unsigned long long* stamps, unsigned long long* evaluated, cudaStream_t st) {
    const size_t sm = sizeof(Stage<CM, kBatchThreads, true>);
    // the evaluated-pair counter is compiled in only when it is asked for
    auto k = evaluated ? k_raster_batch<CM, true> : k_raster_batch<CM, false>;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kBatchThreads, sm);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > total) grid = total;
    if (grid < 1) grid = 1;
    cudaMemsetAsync(counters, 0, sizeof(int) * (size_t)(n_req + 1), st);
    if (stamps) k_stamp<<<1, 1, 0, st>>>(stamps + n_req);
    k<<<(unsigned)grid, kBatchThreads, sm, st>>>(tab, n_req, total, counters, stamps, evaluated);
    return SPLAT_OK;
}

}  // namespace splat

using namespace splat;

extern "C" {

size_t splat_batch_table_bytes(int32_t n_requests) {
    return n_requests > 0 ? sizeof(BatchReqDev) * (size_t)n_requests : 0;
}

splat_status splat_batch_build(const splat_batch_request* reqs, int32_t n_requests, void* table, size_t table_bytes,
                               int64_t* total_items) {
    if (!reqs || n_requests < 1 || n_requests > kMaxBatch || !table || !total_items)
        return record_error(SPLAT_ERR_INVALID_ARG, "splat_batch_build: bad arguments (1..1024 requests)");
    if (table_bytes < splat_batch_table_bytes(n_requests))
        return record_error(SPLAT_ERR_INVALID_ARG, "splat_batch_build: table buffer too small");
    BatchReqDev* tab = reinterpret_cast<BatchReqDev*>(table);
    int64_t items = 0;
    int cm = 0;
    for (int q = 0; q < n_requests; q++) {
        const splat_batch_request& in = reqs[q];
        BatchReqDev d;
        memset(&d, 0, sizeof d);
        const splat_status st =
            frame_sensor_constants(in.group_n_sensors, in.group_sensors, in.group_sensor_index, &d.S);
        if (st != SPLAT_OK) return st;
        if (d.S.tile_w * d.S.tile_h != kBatchThreads * kBatchPX)
            return record_error(SPLAT_ERR_INVALID_ARG, "splat_batch_build: batched tiles must hold 256 rays");
        if (!in.proj.rec || !in.bins.isect_ids || !in.bins.tile_ranges || !in.features || !in.out_feat ||
            in.channels < 1 || in.channels > 32 || in.n < 0)
            return record_error(SPLAT_ERR_INVALID_ARG, "splat_batch_build: bad request buffers");
        if (d.S.kind == SPLAT_SENSOR_LIDAR && (!in.out_range_exp || !in.out_alpha))
            return record_error(SPLAT_ERR_INVALID_ARG, "splat_batch_build: lidar request needs range and alpha");
        d.S.ray_base = 0;
        d.rec = (const float4*)in.proj.rec;
        d.ids = in.bins.isect_ids;
        d.ranges = (const int2*)in.bins.tile_ranges;
        d.n_isect = in.bins.n_isect;
        d.feat = in.features;
        d.n = in.n;
        d.C = in.channels;
        d.sensor_index = in.group_sensor_index;
        d.tiles = d.S.tiles_x * d.S.tiles_y;
        d.item_base = items;
        d.out_feat = in.out_feat;
        d.out_T = in.out_T;
        d.out_range_exp = in.out_range_exp;
        d.out_range_med = in.out_range_med;
        d.out_alpha = in.out_alpha;
        items += d.tiles;
        cm = in.channels > cm ? in.channels : cm;
        memcpy(&tab[q], &d, sizeof d);
    }
    *total_items = items;
    return SPLAT_OK;
}

splat_status splat_stamp(uint64_t* at, void* stream) {
    if (!at) return record_error(SPLAT_ERR_INVALID_ARG, "splat_stamp: NULL");
    k_stamp<<<1, 1, 0, (cudaStream_t)stream>>>((unsigned long long*)at);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return record_error(SPLAT_ERR_CUDA, cudaGetErrorString(e));
    return SPLAT_OK;
}

splat_status splat_render_batch(const void* table, int32_t n_requests, int64_t total_items, int32_t max_channels,
                                int32_t* counters, uint64_t* stamps, uint64_t* evaluated, void* stream) {
    if (!table || n_requests < 1 || n_requests > kMaxBatch || total_items < 0 || !counters)
        return record_error(SPLAT_ERR_INVALID_ARG, "splat_render_batch: bad arguments");
    if (total_items == 0) return SPLAT_OK;
    const BatchReqDev* tab = reinterpret_cast<const BatchReqDev*>(table);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* sp = (unsigned long long*)stamps;
    unsigned long long* ev = (unsigned long long*)evaluated;
    splat_status rc;
    if (max_channels <= 4) rc = launch_batch_t<4>(tab, n_requests, total_items, counters, sp, ev, st);
    else if (max_channels <= 16) rc = launch_batch_t<16>(tab, n_requests, total_items, counters, sp, ev, st);
    else if (max_channels <= 32) rc = launch_batch_t<32>(tab, n_requests, total_items, counters, sp, ev, st);
    else return record_error(SPLAT_ERR_INVALID_ARG, "splat_render_batch: at most 32 channels");
    if (rc != SPLAT_OK) return rc;
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return record_error(SPLAT_ERR_CUDA, cudaGetErrorString(e));
    return SPLAT_OK;
}

}  // extern "C"
