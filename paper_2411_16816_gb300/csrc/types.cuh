// types.cuh -- argument structs shared by the kernels and the C-ABI layer, and the
// launcher declarations of every translation unit.
#pragma once
#include "common.cuh"

namespace splat {

struct GaussIn {
    const float* means;
    const float* scales;
    const float* quats;
    const float* opac;
    const float* vel;
    int64_t n;
};

struct ProjOut {
    float4* rec;
    short4* rect;
    int32_t* n_tiles;
};

struct GradOut {
    float* means;
    float* scales;
    float* quats;
    float* opac;
    float* vel;
    float* sensor;   // optional [sensors][16]: lin_vel, ang_vel, time_offset, -, t, rotation, -
};

// Free lidar rays grouped by tile (App. A.2): the list kernels render these instead of a
// sensor's ray grid, one block per chunk of kListChunk rays of one tile.
constexpr int kListChunk = 256;
struct RayList {
    const float* rays;          // [n_rays][3] phi, omega, t
    const int32_t* ids;         // ray indices grouped by tile of the lidar
    const int2* ranges;         // [tiles] (start, end) into ids
    const int32_t* chunk_base;  // [tiles + 1] first chunk of each tile; [tiles] = number of chunks
    int tiles;
    int sensor;                 // index of the lidar in the frame
    int64_t n_rays = 0;         // rays (and ids) of the list (checked build)
};

struct RasterIn {
    const float4* rec;      // [S][3][n]
    const uint32_t* ids;    // sorted Gaussian indices
    const int2* ranges;     // [total_tiles]
    const float* feat;      // [n][C]
    int64_t n;
    int C;                  // channels (<= the kernel's compile-time maximum CM)
    const float* los_range; // lidar, optional: return range per ray for the line-of-sight term
    float los_eps;
    RayList list;           // list kernels only
    const int64_t* n_isect = nullptr;   // device count of ids (the checked build bounds ranges by it)
};

struct RasterOut {
    float* feat;
    float* T;
    int32_t* last;
    float* range_exp;   // lidar
    float* range_med;   // lidar
    float* alpha;       // lidar
    unsigned long long* evaluated;  // optional: number of (ray, Gaussian) pairs examined
    // optional camera L1 epilogue: loss += scale * sum |F - target|, l1_grad = scale * sign(F - target)
    const float* l1_target;
    float* l1_grad;
    float* l1_loss;
    float l1_scale;
    float* los;             // lidar, optional: line-of-sight term per ray
};

struct RasterGrad {
    const float* T;
    const int32_t* last;
    const float* dfeat;
    const float* dT;       // camera: dL/dT
    const float* drange;   // lidar: dL/d expected range
    const float* dalpha;   // lidar: dL/d (1 - T)
    float4* grad_proj;     // [S][3][n]
    float* dfeatures;      // [n][C]
    const float* dlos;     // lidar, optional: dL/d line-of-sight term
    float* dsensor;        // camera, optional: [sensors][16], entry 6 = dL/d time offset
};

struct BinWorkspace {
    uint32_t* vkeys[2];
    uint32_t* vvals[2];
    int64_t* vis_count;
    int64_t* offsets;        // first row item of each visible pair (depth order)
    uint32_t* row_owner;     // visible pair owning each row block's first row item
    int64_t* n_rows;         // row items (tile rows of the visible pairs' boxes)
    uint32_t* r_key0;        // per row item: tile id of its first listed column
    uint32_t* r_id;          //   Gaussian index
    int32_t* r_wrap;         //   columns before the lidar azimuth wrap (cameras: no wrap)
    int32_t* r_tx;           //   tile columns of its sensor
    int32_t* r_cnt;          //   listed tiles of the row
    int32_t* c_off;          // per row item with tiles (compacted): first output slot
    int32_t* c_row;          //   its row item
    int64_t* slot_total;     // packed (slots, row items with tiles) totals
    int64_t* n_owners;       // row items with tiles
    uint32_t* ikeys[2];
    uint32_t* ivals_tmp;
    uint32_t* first_owner;   // compacted row item owning each emit block's first slot
    uint32_t* hist;
    int64_t* partials;
    size_t bytes;
};

void launch_project(const GaussIn& g, const Frame& fr, const ProjOut& out, cudaStream_t st);
void launch_count_nonfinite(const GaussIn& g, unsigned long long* count, cudaStream_t st);
void launch_project_backward(const GaussIn& g, const Frame& fr, const int32_t* n_tiles, const float4* grad,
                             const GradOut& out, cudaStream_t st);
BinWorkspace carve_workspace(void* base, int64_t pairs, int64_t capacity);
void launch_bin_sort(const Frame& fr, int64_t n, const float4* rec, const short4* rect, const int32_t* n_tiles,
                     int64_t capacity, uint32_t* isect_ids, int2* tile_ranges, int64_t total_tiles,
                     int64_t* n_isect, void* workspace, cudaStream_t st);
bool launch_raster_fwd(bool lidar, int C, int tw, int th, const Frame& fr, int blocks, const RasterIn& in,
                       const RasterOut& out, cudaStream_t st);
bool launch_raster_bwd(bool lidar, int C, int tw, int th, const Frame& fr, int blocks, const RasterIn& in,
                       const RasterGrad& g, bool recompute, cudaStream_t st);
bool launch_raster_list_fwd(int C, const Frame& fr, int blocks, const RasterIn& in, const RasterOut& out,
                            cudaStream_t st);
bool launch_raster_list_bwd(int C, const Frame& fr, int blocks, const RasterIn& in, const RasterGrad& g,
                            bool recompute, cudaStream_t st);
void launch_points_to_rays(const SensorDev& S, const float* points, const float* times, int64_t n, float* rays,
                           float* range, int32_t* tiles, cudaStream_t st);
void launch_bin_rays(const SensorDev& S, const float* rays, int64_t n, int32_t* ids, int2* ranges,
                     int32_t* chunk_base, cudaStream_t st);
void launch_bin_rays_capped(const SensorDev& S, const float* rays, const uint32_t* priority, int64_t n, int cap,
                            int32_t* tmp_ids, int2* tmp_ranges, int32_t* tmp_chunks, int32_t* ids, int2* ranges,
                            int32_t* chunk_base, cudaStream_t st);
bool raster_shape_supported(bool lidar, int tw, int th);
bool raster_channels_supported(int C);
void launch_l1(const float* pred, const float* target, int64_t count, float scale, float* grad, float* loss,
               cudaStream_t st);

struct HeadW {
    const uint16_t* w;   // BF16 W1 | W2 | W3 (row-major [in][out])
    const float* b;      // FP32 b1 | b2 | b3
};
void launch_head_fwd(const float* x, int64_t R, const HeadW& hw, float* out, cudaStream_t st);
bool launch_lidar_fwd_head(int tw, int th, const Frame& fr, int blocks, const RasterIn& in, const RasterOut& out,
                           const HeadW& hw, float* head_out, cudaStream_t st);
void launch_head_train(const float* x, int64_t R, const HeadW& hw, const float* y_int, const float* y_drop, float lam_i,
                       float lam_d, float* grad, float* loss, float* dx, cudaStream_t st);
void launch_head_adam(float* p, const float* g, float* m, float* v, float lr, float beta1, float beta2, float eps,
                      int64_t step, uint16_t* wbf, float* bias, cudaStream_t st);
void launch_head_inputs(const SensorDev& S, const float* feat, int C, float* x, cudaStream_t st);
int head_param_count();

}  // namespace splat
