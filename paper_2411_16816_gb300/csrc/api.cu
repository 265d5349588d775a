// api.cu -- the extern "C" entry points of libsplat (declared in include/splat.h):
// argument checks on the host, the per-frame sensor table, and kernel launches.
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>

#include "status.cuh"
#include "types.cuh"

using namespace splat;

static thread_local std::string g_err;

static splat_status fail(splat_status code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
static splat_status fail(splat_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

static splat_status check_launch(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(SPLAT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    g_err.clear();
    return SPLAT_OK;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Tiles the binning supports: 64 to 512 rays, both sides powers of two.  The per-frame
// raster entry points have kernels for a subset (raster_shape_supported); the batched
// persistent launch takes any 256-ray tile.
static bool tile_shape_ok(int tw, int th) {
    auto pow2 = [](int v) { return v >= 1 && (v & (v - 1)) == 0; };
    const int r = tw * th;
    return pow2(tw) && pow2(th) && r >= 64 && r <= 512;
}

// Per-sensor constants and the frame's tile / block / ray numbering.
static splat_status build_frame(int32_t n_sensors, const splat_sensor* sensors, Frame& fr, int64_t* total_tiles) {
    if (n_sensors < 1 || n_sensors > kMaxSensors)
        return fail(SPLAT_ERR_INVALID_ARG, "n_sensors must be in [1, %d], got %d", kMaxSensors, n_sensors);
    if (!sensors) return fail(SPLAT_ERR_INVALID_ARG, "sensors is NULL");
    memset(&fr, 0, sizeof fr);
    fr.n_sensors = n_sensors;
    int64_t tile_base = 0, cam_blocks = 0, lid_blocks = 0, cam_rays = 0, lid_rays = 0;
    for (int s = 0; s < n_sensors; s++) {
        const splat_sensor& in = sensors[s];
        SensorDev& d = fr.s[s];
        d.kind = in.kind;
        memcpy(d.R, in.R, sizeof d.R);
        memcpy(d.t, in.t, sizeof d.t);
        memcpy(d.v, in.lin_vel, sizeof d.v);
        memcpy(d.w, in.ang_vel, sizeof d.w);
        d.tile_w = in.tile_w;
        d.tile_h = in.tile_h;
        d.eps = in.eps2d;
        if (!(in.eps2d >= 0.f)) return fail(SPLAT_ERR_INVALID_ARG, "sensor %d: eps2d must be >= 0", s);
        if (in.support & ~7)
            return fail(SPLAT_ERR_INVALID_ARG,
                        "sensor %d: support flags are 1 (opacity-aware), 2 (sweep times) and 4 (camera tile cull)", s);
        if ((in.support & 2) && (in.kind != SPLAT_SENSOR_LIDAR || in.rays))
            return fail(SPLAT_ERR_INVALID_ARG, "sensor %d: sweep-time margins need a lidar on its regular ray grid", s);
        d.support = in.kind == SPLAT_SENSOR_CAMERA ? in.support : (in.support & 3);   // the cull is for cameras
        const bool lidar = in.kind == SPLAT_SENSOR_LIDAR;
        if (in.kind != SPLAT_SENSOR_CAMERA && !lidar) return fail(SPLAT_ERR_INVALID_ARG, "sensor %d: bad kind", s);
        if (!tile_shape_ok(in.tile_w, in.tile_h))
            return fail(SPLAT_ERR_INVALID_ARG, "sensor %d: unsupported tile %dx%d", s, in.tile_w, in.tile_h);
        int64_t rays;
        if (!lidar) {
            if (in.width < 1 || in.height < 1 || !(in.fx > 0.f) || !(in.fy > 0.f))
                return fail(SPLAT_ERR_INVALID_ARG, "camera %d: bad size or focal length", s);
            d.width = in.width;
            d.height = in.height;
            d.fx = in.fx;
            d.fy = in.fy;
            d.cx = in.cx;
            d.cy = in.cy;
            d.rs = in.rs_time;
            d.dt = in.time_offset;
            d.near_plane = in.near_plane;
            d.lim_x = 1.3f * 0.5f * (float)in.width / in.fx;
            d.lim_y = 1.3f * 0.5f * (float)in.height / in.fy;
            d.tiles_x = (in.width + in.tile_w - 1) / in.tile_w;
            d.tiles_y = (in.height + in.tile_h - 1) / in.tile_h;
            rays = (int64_t)in.width * in.height;
        } else {
            if (in.n_beams < 2 || in.n_az < 1 || !in.beam_elev || !(in.az_res > 0.f))
                return fail(SPLAT_ERR_INVALID_ARG, "lidar %d: bad beams/azimuth/elevations", s);
            if (in.n_beams % in.tile_h != 0)
                return fail(SPLAT_ERR_INVALID_ARG, "lidar %d: n_beams %d not a multiple of tile_h %d", s, in.n_beams,
                            in.tile_h);
            if (std::fabs((double)in.n_az * in.az_res - 2.0 * M_PI) > 1e-3)
                return fail(SPLAT_ERR_INVALID_ARG, "lidar %d: n_az * az_res must cover 2 pi", s);
            d.nb = in.n_beams;
            d.naz = in.n_az;
            d.elev = in.beam_elev;
            d.rays = in.rays;
            d.az_res = in.az_res;
            d.sweep = in.sweep_time;
            d.rmin = in.r_min;
            d.tiles_x = (in.n_az + in.tile_w - 1) / in.tile_w;
            d.tiles_y = in.n_beams / in.tile_h;
            d.wphi = (float)in.tile_w * in.az_res;
            d.phimax = (float)d.tiles_x * d.wphi;
            rays = (int64_t)in.n_beams * in.n_az;
        }
        const int64_t tiles = (int64_t)d.tiles_x * d.tiles_y;
        d.tile_base = (int)tile_base;
        tile_base += tiles;
        if (!lidar) {
            d.block_base = (int)cam_blocks;
            d.ray_base = (int)cam_rays;
            cam_blocks += tiles;
            cam_rays += rays;
            fr.cam_sensors[fr.n_cams++] = s;
        } else {
            d.block_base = (int)lid_blocks;
            d.ray_base = (int)lid_rays;
            lid_blocks += tiles;
            lid_rays += rays;
            fr.lid_sensors[fr.n_lids++] = s;
        }
        if (tile_base > (int64_t)1 << 30 || cam_rays > (int64_t)1 << 31 || lid_rays > (int64_t)1 << 31)
            return fail(SPLAT_ERR_INVALID_ARG, "frame too large");
    }
    fr.n_cam_blocks = (int)cam_blocks;
    fr.n_lid_blocks = (int)lid_blocks;
    if (total_tiles) *total_tiles = tile_base;
    return SPLAT_OK;
}

static splat_status check_gaussians(const splat_gaussians* g, bool need_features) {
    if (!g) return fail(SPLAT_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->n < 0) return fail(SPLAT_ERR_INVALID_ARG, "n < 0");
    if (g->n > 0 && (!g->means || !g->scales || !g->quats || !g->opacities))
        return fail(SPLAT_ERR_INVALID_ARG, "gaussian parameter pointer is NULL");
    if (g->n > 0 && !aligned16(g->quats)) return fail(SPLAT_ERR_INVALID_ARG, "quats must be 16-byte aligned");
    if (need_features) {
        if (!raster_channels_supported(g->channels))
            return fail(SPLAT_ERR_INVALID_ARG, "channels must be in [1, 32], got %d", g->channels);
        if (g->n > 0 && !g->features) return fail(SPLAT_ERR_INVALID_ARG, "features is NULL");
        if ((g->channels & 3) == 0 && !aligned16(g->features))
            return fail(SPLAT_ERR_INVALID_ARG, "features must be 16-byte aligned");
    }
    return SPLAT_OK;
}

static splat_status check_proj(const splat_projected& p) {
    if (!p.rec || !p.rect || !p.n_tiles) return fail(SPLAT_ERR_INVALID_ARG, "projected buffer is NULL");
    if (!aligned16(p.rec) || ((uintptr_t)p.rect & 7u)) return fail(SPLAT_ERR_INVALID_ARG, "projected misaligned");
    return SPLAT_OK;
}

static GaussIn gauss_in(const splat_gaussians* g) {
    return GaussIn{g->means, g->scales, g->quats, g->opacities, g->velocities, g->n};
}

extern "C" {

splat_status splat_frame_layout(int32_t n_sensors, const splat_sensor* sensors, int64_t* total_tiles,
                                int64_t* tiles_out, int64_t* rays_out) {
    Frame fr;
    const splat_status st = build_frame(n_sensors, sensors, fr, total_tiles);
    if (st != SPLAT_OK) return st;
    for (int s = 0; s < n_sensors; s++) {
        const SensorDev& d = fr.s[s];
        if (tiles_out) tiles_out[s] = (int64_t)d.tiles_x * d.tiles_y;
        if (rays_out) rays_out[s] = d.kind == SPLAT_SENSOR_CAMERA ? (int64_t)d.width * d.height : (int64_t)d.nb * d.naz;
    }
    return SPLAT_OK;
}

splat_status splat_workspace_size(int64_t n, int32_t n_sensors, const splat_sensor* sensors, int64_t capacity,
                                  size_t* bytes) {
    Frame fr;
    const splat_status st = build_frame(n_sensors, sensors, fr, nullptr);
    if (st != SPLAT_OK) return st;
    if (!bytes || n < 0 || capacity < 0) return fail(SPLAT_ERR_INVALID_ARG, "bad workspace query");
    *bytes = carve_workspace(nullptr, (int64_t)n_sensors * n, capacity).bytes;
    return SPLAT_OK;
}

splat_status splat_project(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                           splat_projected proj, void* stream) {
    splat_status st = check_gaussians(g, false);
    if (st != SPLAT_OK) return st;
    Frame fr;
    if ((st = build_frame(n_sensors, sensors, fr, nullptr)) != SPLAT_OK) return st;
    if ((st = check_proj(proj)) != SPLAT_OK) return st;
    if ((int64_t)n_sensors * g->n >= ((int64_t)1 << 32))
        return fail(SPLAT_ERR_INVALID_ARG, "n_sensors * n must be below 2^32");
    launch_project(gauss_in(g), fr, ProjOut{(float4*)proj.rec, (short4*)proj.rect, proj.n_tiles},
                   (cudaStream_t)stream);
    return check_launch("splat_project");
}

splat_status splat_count_nonfinite(const splat_gaussians* g, int64_t* count, void* stream) {
    splat_status st = check_gaussians(g, false);
    if (st != SPLAT_OK) return st;
    if (!count || ((uintptr_t)count & 7u)) return fail(SPLAT_ERR_INVALID_ARG, "count is NULL or misaligned");
    launch_count_nonfinite(gauss_in(g), reinterpret_cast<unsigned long long*>(count), (cudaStream_t)stream);
    return check_launch("splat_count_nonfinite");
}

splat_status splat_bin_sort(int64_t n, int32_t n_sensors, const splat_sensor* sensors, splat_projected proj,
                            int64_t capacity, splat_bins bins, void* workspace, size_t workspace_bytes,
                            void* stream) {
    Frame fr;
    int64_t total_tiles = 0;
    splat_status st = build_frame(n_sensors, sensors, fr, &total_tiles);
    if (st != SPLAT_OK) return st;
    if ((st = check_proj(proj)) != SPLAT_OK) return st;
    if (n < 0 || capacity < 0 || capacity >= ((int64_t)1 << 31))
        return fail(SPLAT_ERR_INVALID_ARG, "capacity must be in [0, 2^31)");
    if ((int64_t)n_sensors * n >= ((int64_t)1 << 32))
        return fail(SPLAT_ERR_INVALID_ARG, "n_sensors * n must be below 2^32");
    if (!bins.isect_ids || !bins.tile_ranges || !bins.n_isect || !workspace)
        return fail(SPLAT_ERR_INVALID_ARG, "bins or workspace pointer is NULL");
    if (((uintptr_t)bins.tile_ranges & 7u) || ((uintptr_t)bins.n_isect & 7u) || ((uintptr_t)workspace & 255u))
        return fail(SPLAT_ERR_INVALID_ARG, "bins or workspace misaligned");
    const size_t need = carve_workspace(nullptr, (int64_t)n_sensors * n, capacity).bytes;
    if (workspace_bytes < need)
        return fail(SPLAT_ERR_INVALID_ARG, "workspace too small: %zu < %zu bytes", workspace_bytes, need);
    launch_bin_sort(fr, n, (const float4*)proj.rec, (const short4*)proj.rect, proj.n_tiles, capacity, bins.isect_ids,
                    (int2*)bins.tile_ranges, total_tiles, bins.n_isect, workspace, (cudaStream_t)stream);
    return check_launch("splat_bin_sort");
}

splat_status splat_bin_sort_backward(void) { return SPLAT_OK; }

static splat_status render_common(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                                  splat_projected proj, splat_bins bins, Frame& fr, bool lidar, int& tw, int& th) {
    splat_status st = check_gaussians(g, true);
    if (st != SPLAT_OK) return st;
    if ((st = build_frame(n_sensors, sensors, fr, nullptr)) != SPLAT_OK) return st;
    if ((st = check_proj(proj)) != SPLAT_OK) return st;
    if (!bins.isect_ids || !bins.tile_ranges) return fail(SPLAT_ERR_INVALID_ARG, "bins pointer is NULL");
    tw = th = 0;
    const int nk = lidar ? fr.n_lids : fr.n_cams;
    const int* list = lidar ? fr.lid_sensors : fr.cam_sensors;
    for (int k = 0; k < nk; k++) {
        const SensorDev& d = fr.s[list[k]];
        if (k == 0) {
            tw = d.tile_w;
            th = d.tile_h;
        } else if (d.tile_w != tw || d.tile_h != th) {
            return fail(SPLAT_ERR_INVALID_ARG, "all %s sensors of a frame must share one tile shape",
                        lidar ? "lidar" : "camera");
        }
    }
    return SPLAT_OK;
}

splat_status splat_render_camera(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                                 splat_projected proj, splat_bins bins, float* out_feat, float* out_T,
                                 int32_t* out_last, uint64_t* evaluated, void* stream) {
    Frame fr;
    int tw, th;
    splat_status st = render_common(g, n_sensors, sensors, proj, bins, fr, false, tw, th);
    if (st != SPLAT_OK) return st;
    if (fr.n_cams == 0) return SPLAT_OK;
    if (!out_feat) return fail(SPLAT_ERR_INVALID_ARG, "out_feat is NULL");
    if ((g->channels & 3) == 0 && !aligned16(out_feat)) return fail(SPLAT_ERR_INVALID_ARG, "out_feat misaligned");
    RasterIn in{(const float4*)proj.rec, bins.isect_ids, (const int2*)bins.tile_ranges, g->features, g->n,
                g->channels};
    in.n_isect = bins.n_isect;
    RasterOut out{out_feat, out_T, out_last, nullptr, nullptr, nullptr, (unsigned long long*)evaluated};
    if (!launch_raster_fwd(false, g->channels, tw, th, fr, fr.n_cam_blocks, in, out, (cudaStream_t)stream))
        return fail(SPLAT_ERR_INVALID_ARG, "unsupported camera configuration");
    return check_launch("splat_render_camera");
}

splat_status splat_render_camera_l1(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                                    splat_projected proj, splat_bins bins, const float* target, float scale,
                                    float* out_feat, float* out_T, int32_t* out_last, float* grad_feat, float* loss,
                                    uint64_t* evaluated, void* stream) {
    Frame fr;
    int tw, th;
    splat_status st = render_common(g, n_sensors, sensors, proj, bins, fr, false, tw, th);
    if (st != SPLAT_OK) return st;
    if (fr.n_cams == 0) return SPLAT_OK;
    if (!target || !grad_feat || !loss) return fail(SPLAT_ERR_INVALID_ARG, "target, grad_feat and loss are required");
    if ((g->channels & 3) == 0 &&
        !(aligned16(target) && aligned16(grad_feat) && (!out_feat || aligned16(out_feat))))
        return fail(SPLAT_ERR_INVALID_ARG, "target, grad_feat or out_feat misaligned");
    RasterIn in{(const float4*)proj.rec, bins.isect_ids, (const int2*)bins.tile_ranges, g->features, g->n,
                g->channels};
    in.n_isect = bins.n_isect;
    RasterOut out{out_feat, out_T, out_last, nullptr, nullptr, nullptr, (unsigned long long*)evaluated,
                  target, grad_feat, loss, scale};
    if (!launch_raster_fwd(false, g->channels, tw, th, fr, fr.n_cam_blocks, in, out, (cudaStream_t)stream))
        return fail(SPLAT_ERR_INVALID_ARG, "unsupported camera configuration");
    return check_launch("splat_render_camera_l1");
}

splat_status splat_sync_status(void* stream) {
    const cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return fail(SPLAT_ERR_CUDA, "%s", cudaGetErrorString(e));
    const cudaError_t e2 = cudaGetLastError();
    if (e2 != cudaSuccess) return fail(SPLAT_ERR_CUDA, "%s", cudaGetErrorString(e2));
    uint32_t bits = 0, site = 0;
    take_all_status(&bits, &site);
    if (bits & kStatusTimeout)
        return fail(SPLAT_ERR_TIMEOUT, "a bounded wait for tensor-core work ran out (site %u)", site);
    if (bits & kStatusBounds)
        return fail(SPLAT_ERR_BOUNDS, "checked build: an out-of-bounds index was skipped (site %u)", site);
    return SPLAT_OK;
}

int32_t splat_build_flags(void) {
#ifdef SPLAT_CHECKED
    return 1;
#else
    return 0;
#endif
}

static splat_status render_lidar_impl(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                                      splat_projected proj, splat_bins bins, float* out_feat, float* out_range_exp,
                                      float* out_range_med, float* out_alpha, float* out_T, int32_t* out_last,
                                      const splat_los* los, float* out_los, uint64_t* evaluated, void* stream,
                                      const char* name) {
    Frame fr;
    int tw, th;
    splat_status st = render_common(g, n_sensors, sensors, proj, bins, fr, true, tw, th);
    if (st != SPLAT_OK) return st;
    if (fr.n_lids == 0) return SPLAT_OK;
    if (!out_feat || !out_range_exp || !out_alpha)
        return fail(SPLAT_ERR_INVALID_ARG, "out_feat, out_range_exp and out_alpha are required");
    if ((g->channels & 3) == 0 && !aligned16(out_feat)) return fail(SPLAT_ERR_INVALID_ARG, "out_feat misaligned");
    if (los && (!los->target_range || !out_los || !(los->eps >= 0.f)))
        return fail(SPLAT_ERR_INVALID_ARG, "%s: los.target_range and out_los are required, los.eps >= 0", name);
    RasterIn in{(const float4*)proj.rec, bins.isect_ids, (const int2*)bins.tile_ranges, g->features, g->n,
                g->channels, los ? los->target_range : nullptr, los ? los->eps : 0.f};
    in.n_isect = bins.n_isect;
    RasterOut out{out_feat, out_T, out_last, out_range_exp, out_range_med, out_alpha,
                  (unsigned long long*)evaluated};
    out.los = los ? out_los : nullptr;
    if (!launch_raster_fwd(true, g->channels, tw, th, fr, fr.n_lid_blocks, in, out, (cudaStream_t)stream))
        return fail(SPLAT_ERR_INVALID_ARG, "unsupported lidar configuration");
    return check_launch(name);
}


splat_status splat_render_lidar(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                                splat_projected proj, splat_bins bins, float* out_feat, float* out_range_exp,
                                float* out_range_med, float* out_alpha, float* out_T, int32_t* out_last,
                                uint64_t* evaluated, void* stream) {
    return render_lidar_impl(g, n_sensors, sensors, proj, bins, out_feat, out_range_exp, out_range_med, out_alpha,
                             out_T, out_last, nullptr, nullptr, evaluated, stream, "splat_render_lidar");
}

splat_status splat_render_lidar_los(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                                    splat_projected proj, splat_bins bins, float* out_feat, float* out_range_exp,
                                    float* out_range_med, float* out_alpha, float* out_T, int32_t* out_last,
                                    splat_los los, float* out_los, uint64_t* evaluated, void* stream) {
    return render_lidar_impl(g, n_sensors, sensors, proj, bins, out_feat, out_range_exp, out_range_med, out_alpha,
                             out_T, out_last, &los, out_los, evaluated, stream, "splat_render_lidar_los");
}

splat_status splat_render_lidar_head(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                                     splat_projected proj, splat_bins bins, float* out_feat, float* out_range_exp,
                                     float* out_range_med, float* out_alpha, float* out_T, int32_t* out_last,
                                     const uint16_t* head_w, const float* head_b, float* out_head, void* stream) {
    Frame fr;
    int tw, th;
    splat_status st = render_common(g, n_sensors, sensors, proj, bins, fr, true, tw, th);
    if (st != SPLAT_OK) return st;
    if (fr.n_lids == 0) return SPLAT_OK;
    if (g->channels != 29) return fail(SPLAT_ERR_INVALID_ARG, "splat_render_lidar_head: channels must be 29");
    if (tw != 32 || th != 8) return fail(SPLAT_ERR_INVALID_ARG, "splat_render_lidar_head: the lidar tile must be 32 x 8");
    if (!out_range_exp || !out_alpha || !head_w || !head_b || !out_head)
        return fail(SPLAT_ERR_INVALID_ARG, "out_range_exp, out_alpha, head_w, head_b and out_head are required");
    if (((uintptr_t)out_head & 7u) || ((uintptr_t)head_w & 3u))
        return fail(SPLAT_ERR_INVALID_ARG, "out_head or head_w misaligned");
    RasterIn in{(const float4*)proj.rec, bins.isect_ids, (const int2*)bins.tile_ranges, g->features, g->n,
                g->channels};
    in.n_isect = bins.n_isect;
    RasterOut out{out_feat, out_T, out_last, out_range_exp, out_range_med, out_alpha, nullptr};
    if (!launch_lidar_fwd_head(tw, th, fr, fr.n_lid_blocks, in, out, HeadW{head_w, head_b}, out_head,
                               (cudaStream_t)stream))
        return fail(SPLAT_ERR_INVALID_ARG, "unsupported lidar configuration");
    return check_launch("splat_render_lidar_head");
}

splat_status splat_render_camera_backward(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                                          splat_projected proj, splat_bins bins, const float* out_T,
                                          const int32_t* out_last, const float* dL_dfeat, const float* dL_dT,
                                          float* grad_proj, float* dL_dfeatures, float* dL_dsensors, void* stream) {
    Frame fr;
    int tw, th;
    splat_status st = render_common(g, n_sensors, sensors, proj, bins, fr, false, tw, th);
    if (st != SPLAT_OK) return st;
    if (fr.n_cams == 0) return SPLAT_OK;
    if (!dL_dfeat || !grad_proj || !dL_dfeatures) return fail(SPLAT_ERR_INVALID_ARG, "gradient pointer is NULL");
    if ((out_T == nullptr) != (out_last == nullptr))
        return fail(SPLAT_ERR_INVALID_ARG, "out_T and out_last must both be given or both be NULL");
    if (!aligned16(grad_proj) || ((g->channels & 3) == 0 && !aligned16(dL_dfeatures)))
        return fail(SPLAT_ERR_INVALID_ARG, "gradient buffers misaligned");
    RasterIn in{(const float4*)proj.rec, bins.isect_ids, (const int2*)bins.tile_ranges, g->features, g->n,
                g->channels};
    in.n_isect = bins.n_isect;
    RasterGrad gr{out_T, out_last, dL_dfeat, dL_dT, nullptr, nullptr, (float4*)grad_proj, dL_dfeatures, nullptr,
                  dL_dsensors};
    if (!launch_raster_bwd(false, g->channels, tw, th, fr, fr.n_cam_blocks, in, gr, out_T == nullptr,
                           (cudaStream_t)stream))
        return fail(SPLAT_ERR_INVALID_ARG, "unsupported camera configuration");
    return check_launch("splat_render_camera_backward");
}

static splat_status render_lidar_backward_impl(const splat_gaussians* g, int32_t n_sensors,
                                               const splat_sensor* sensors, splat_projected proj, splat_bins bins,
                                               const float* out_T, const int32_t* out_last, const float* dL_dfeat,
                                               const float* dL_drange_exp, const float* dL_dalpha,
                                               const splat_los* los, const float* dL_dlos, float* grad_proj,
                                               float* dL_dfeatures, void* stream, const char* name) {
    Frame fr;
    int tw, th;
    splat_status st = render_common(g, n_sensors, sensors, proj, bins, fr, true, tw, th);
    if (st != SPLAT_OK) return st;
    if (fr.n_lids == 0) return SPLAT_OK;
    if (!dL_dfeat || !grad_proj || !dL_dfeatures) return fail(SPLAT_ERR_INVALID_ARG, "gradient pointer is NULL");
    if ((out_T == nullptr) != (out_last == nullptr))
        return fail(SPLAT_ERR_INVALID_ARG, "out_T and out_last must both be given or both be NULL");
    if (!aligned16(grad_proj) || ((g->channels & 3) == 0 && !aligned16(dL_dfeatures)))
        return fail(SPLAT_ERR_INVALID_ARG, "gradient buffers misaligned");
    if (los && (!los->target_range || !dL_dlos || !(los->eps >= 0.f)))
        return fail(SPLAT_ERR_INVALID_ARG, "%s: los.target_range and dL_dlos are required, los.eps >= 0", name);
    RasterIn in{(const float4*)proj.rec, bins.isect_ids, (const int2*)bins.tile_ranges, g->features, g->n,
                g->channels, los ? los->target_range : nullptr, los ? los->eps : 0.f};
    in.n_isect = bins.n_isect;
    RasterGrad gr{out_T, out_last, dL_dfeat, nullptr, dL_drange_exp, dL_dalpha, (float4*)grad_proj, dL_dfeatures,
                  los ? dL_dlos : nullptr};
    if (!launch_raster_bwd(true, g->channels, tw, th, fr, fr.n_lid_blocks, in, gr, out_T == nullptr,
                           (cudaStream_t)stream))
        return fail(SPLAT_ERR_INVALID_ARG, "unsupported lidar configuration");
    return check_launch(name);
}

splat_status splat_render_lidar_backward(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                                         splat_projected proj, splat_bins bins, const float* out_T,
                                         const int32_t* out_last, const float* dL_dfeat,
                                         const float* dL_drange_exp, const float* dL_dalpha, float* grad_proj,
                                         float* dL_dfeatures, void* stream) {
    return render_lidar_backward_impl(g, n_sensors, sensors, proj, bins, out_T, out_last, dL_dfeat, dL_drange_exp,
                                      dL_dalpha, nullptr, nullptr, grad_proj, dL_dfeatures, stream,
                                      "splat_render_lidar_backward");
}

splat_status splat_render_lidar_backward_los(const splat_gaussians* g, int32_t n_sensors,
                                             const splat_sensor* sensors, splat_projected proj, splat_bins bins,
                                             const float* out_T, const int32_t* out_last, const float* dL_dfeat,
                                             const float* dL_drange_exp, const float* dL_dalpha, splat_los los,
                                             const float* dL_dlos, float* grad_proj, float* dL_dfeatures,
                                             void* stream) {
    return render_lidar_backward_impl(g, n_sensors, sensors, proj, bins, out_T, out_last, dL_dfeat, dL_drange_exp,
                                      dL_dalpha, &los, dL_dlos, grad_proj, dL_dfeatures, stream,
                                      "splat_render_lidar_backward_los");
}

// ---- free lidar rays (App. A.2) ------------------------------------------------------

static splat_status lidar_of(int32_t n_sensors, const splat_sensor* sensors, int32_t lidar, Frame& fr,
                             const char* name) {
    splat_status st = build_frame(n_sensors, sensors, fr, nullptr);
    if (st != SPLAT_OK) return st;
    if (lidar < 0 || lidar >= n_sensors || fr.s[lidar].kind != SPLAT_SENSOR_LIDAR)
        return fail(SPLAT_ERR_INVALID_ARG, "%s: sensor %d is not a lidar of the table", name, lidar);
    return SPLAT_OK;
}

static splat_status check_ray_bins(const splat_ray_bins& b, int64_t n_rays, const char* name) {
    if (n_rays < 0 || n_rays > INT32_MAX) return fail(SPLAT_ERR_INVALID_ARG, "%s: n_rays out of range", name);
    if ((n_rays > 0 && !b.ray_ids) || !b.tile_ranges || !b.chunk_base)
        return fail(SPLAT_ERR_INVALID_ARG, "%s: ray bins pointer is NULL", name);
    if (((uintptr_t)b.tile_ranges & 7u) != 0)
        return fail(SPLAT_ERR_INVALID_ARG, "%s: tile_ranges must be 8-byte aligned", name);
    return SPLAT_OK;
}

splat_status splat_lidar_points_to_rays(int32_t n_sensors, const splat_sensor* sensors, int32_t lidar,
                                        const float* points, const float* times, int64_t n_points, float* rays,
                                        float* ranges, int32_t* tiles, void* stream) {
    Frame fr;
    splat_status st = lidar_of(n_sensors, sensors, lidar, fr, "splat_lidar_points_to_rays");
    if (st != SPLAT_OK) return st;
    if (n_points < 0 || n_points > INT32_MAX) return fail(SPLAT_ERR_INVALID_ARG, "n_points out of range");
    if (n_points == 0) return SPLAT_OK;
    if (!points || !times || !rays || !ranges)
        return fail(SPLAT_ERR_INVALID_ARG, "splat_lidar_points_to_rays: points, times, rays and ranges are required");
    launch_points_to_rays(fr.s[lidar], points, times, n_points, rays, ranges, tiles, (cudaStream_t)stream);
    return check_launch("splat_lidar_points_to_rays");
}

splat_status splat_lidar_bin_rays(int32_t n_sensors, const splat_sensor* sensors, int32_t lidar, const float* rays,
                                  int64_t n_rays, splat_ray_bins bins, void* stream) {
    Frame fr;
    splat_status st = lidar_of(n_sensors, sensors, lidar, fr, "splat_lidar_bin_rays");
    if (st != SPLAT_OK) return st;
    if ((st = check_ray_bins(bins, n_rays, "splat_lidar_bin_rays")) != SPLAT_OK) return st;
    if (n_rays > 0 && !rays) return fail(SPLAT_ERR_INVALID_ARG, "splat_lidar_bin_rays: rays is NULL");
    launch_bin_rays(fr.s[lidar], rays, n_rays, bins.ray_ids, (int2*)bins.tile_ranges, bins.chunk_base,
                    (cudaStream_t)stream);
    return check_launch("splat_lidar_bin_rays");
}

splat_status splat_lidar_bin_rays_capped(int32_t n_sensors, const splat_sensor* sensors, int32_t lidar,
                                         const float* rays, const uint32_t* priority, int64_t n_rays, int32_t cap,
                                         splat_ray_bins scratch, splat_ray_bins bins, void* stream) {
    const char* name = "splat_lidar_bin_rays_capped";
    Frame fr;
    splat_status st = lidar_of(n_sensors, sensors, lidar, fr, name);
    if (st != SPLAT_OK) return st;
    if ((st = check_ray_bins(bins, n_rays, name)) != SPLAT_OK) return st;
    if ((st = check_ray_bins(scratch, n_rays, name)) != SPLAT_OK) return st;
    if (cap < 1) return fail(SPLAT_ERR_INVALID_ARG, "%s: cap must be >= 1", name);
    if (n_rays > 0 && (!rays || !priority)) return fail(SPLAT_ERR_INVALID_ARG, "%s: rays and priority are required", name);
    launch_bin_rays_capped(fr.s[lidar], rays, priority, n_rays, cap, scratch.ray_ids, (int2*)scratch.tile_ranges,
                           scratch.chunk_base, bins.ray_ids, (int2*)bins.tile_ranges, bins.chunk_base,
                           (cudaStream_t)stream);
    return check_launch(name);
}

// Free-ray raster input: the frame's lists plus the lidar's binned rays; the grid bounds
// the number of 256-ray chunks (sum of ceil(count / 256) <= n_rays / 256 + tiles).
static splat_status list_input(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                               int32_t lidar, splat_projected proj, splat_bins bins, const float* rays,
                               int64_t n_rays, const splat_ray_bins& rb, Frame& fr, RasterIn& in, int& blocks,
                               const char* name) {
    int tw, th;
    splat_status st = render_common(g, n_sensors, sensors, proj, bins, fr, true, tw, th);
    if (st != SPLAT_OK) return st;
    if (lidar < 0 || lidar >= n_sensors || fr.s[lidar].kind != SPLAT_SENSOR_LIDAR)
        return fail(SPLAT_ERR_INVALID_ARG, "%s: sensor %d is not a lidar of the table", name, lidar);
    if ((st = check_ray_bins(rb, n_rays, name)) != SPLAT_OK) return st;
    if (n_rays > 0 && !rays) return fail(SPLAT_ERR_INVALID_ARG, "%s: rays is NULL", name);
    const SensorDev& S = fr.s[lidar];
    if (S.support & 2)
        return fail(SPLAT_ERR_INVALID_ARG, "%s: the lidar's lists assume its grid's ray times (support flag 2)", name);
    const int tiles = S.tiles_x * S.tiles_y;
    const int64_t b = (n_rays + kListChunk - 1) / kListChunk + tiles;
    if (b > INT32_MAX) return fail(SPLAT_ERR_INVALID_ARG, "%s: too many rays", name);
    blocks = n_rays > 0 ? (int)b : 0;
    in = RasterIn{(const float4*)proj.rec, bins.isect_ids, (const int2*)bins.tile_ranges, g->features, g->n,
                  g->channels};
    in.n_isect = bins.n_isect;
    in.list = RayList{rays, rb.ray_ids, (const int2*)rb.tile_ranges, rb.chunk_base, tiles, lidar, n_rays};
    return SPLAT_OK;
}

splat_status splat_render_lidar_rays(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                                     int32_t lidar, splat_projected proj, splat_bins bins, const float* rays,
                                     int64_t n_rays, splat_ray_bins ray_bins, float* out_feat,
                                     float* out_range_exp, float* out_range_med, float* out_alpha, float* out_T,
                                     int32_t* out_last, const splat_los* los, float* out_los, void* stream) {
    const char* name = "splat_render_lidar_rays";
    Frame fr;
    RasterIn in;
    int blocks = 0;
    splat_status st = list_input(g, n_sensors, sensors, lidar, proj, bins, rays, n_rays, ray_bins, fr, in, blocks,
                                 name);
    if (st != SPLAT_OK) return st;
    if (n_rays == 0) return SPLAT_OK;
    if (!out_feat || !out_range_exp || !out_alpha)
        return fail(SPLAT_ERR_INVALID_ARG, "%s: out_feat, out_range_exp and out_alpha are required", name);
    if ((g->channels & 3) == 0 && !aligned16(out_feat)) return fail(SPLAT_ERR_INVALID_ARG, "out_feat misaligned");
    if (los && (!los->target_range || !out_los || !(los->eps >= 0.f)))
        return fail(SPLAT_ERR_INVALID_ARG, "%s: los.target_range and out_los are required, los.eps >= 0", name);
    in.los_range = los ? los->target_range : nullptr;
    in.los_eps = los ? los->eps : 0.f;
    RasterOut out{out_feat, out_T, out_last, out_range_exp, out_range_med, out_alpha, nullptr};
    out.los = los ? out_los : nullptr;
    if (!launch_raster_list_fwd(g->channels, fr, blocks, in, out, (cudaStream_t)stream))
        return fail(SPLAT_ERR_INVALID_ARG, "%s: unsupported configuration", name);
    return check_launch(name);
}

splat_status splat_render_lidar_rays_backward(const splat_gaussians* g, int32_t n_sensors,
                                              const splat_sensor* sensors, int32_t lidar, splat_projected proj,
                                              splat_bins bins, const float* rays, int64_t n_rays,
                                              splat_ray_bins ray_bins, const float* out_T, const int32_t* out_last,
                                              const float* dL_dfeat, const float* dL_drange_exp,
                                              const float* dL_dalpha, const splat_los* los, const float* dL_dlos,
                                              float* grad_proj, float* dL_dfeatures, void* stream) {
    const char* name = "splat_render_lidar_rays_backward";
    Frame fr;
    RasterIn in;
    int blocks = 0;
    splat_status st = list_input(g, n_sensors, sensors, lidar, proj, bins, rays, n_rays, ray_bins, fr, in, blocks,
                                 name);
    if (st != SPLAT_OK) return st;
    if (n_rays == 0) return SPLAT_OK;
    if (!dL_dfeat || !grad_proj || !dL_dfeatures) return fail(SPLAT_ERR_INVALID_ARG, "gradient pointer is NULL");
    if ((out_T == nullptr) != (out_last == nullptr))
        return fail(SPLAT_ERR_INVALID_ARG, "out_T and out_last must both be given or both be NULL");
    if (!aligned16(grad_proj) || ((g->channels & 3) == 0 && !aligned16(dL_dfeatures)))
        return fail(SPLAT_ERR_INVALID_ARG, "gradient buffers misaligned");
    if ((los != nullptr) != (dL_dlos != nullptr) || (los && (!los->target_range || !(los->eps >= 0.f))))
        return fail(SPLAT_ERR_INVALID_ARG, "%s: los and dL_dlos go together, los.eps >= 0", name);
    in.los_range = los ? los->target_range : nullptr;
    in.los_eps = los ? los->eps : 0.f;
    RasterGrad gr{out_T, out_last, dL_dfeat, nullptr, dL_drange_exp, dL_dalpha, (float4*)grad_proj, dL_dfeatures,
                  dL_dlos};
    if (!launch_raster_list_bwd(g->channels, fr, blocks, in, gr, out_T == nullptr, (cudaStream_t)stream))
        return fail(SPLAT_ERR_INVALID_ARG, "%s: unsupported configuration", name);
    return check_launch(name);
}

splat_status splat_project_backward(const splat_gaussians* g, int32_t n_sensors, const splat_sensor* sensors,
                                    splat_projected proj, const float* grad_proj, float* dL_dmeans,
                                    float* dL_dscales, float* dL_dquats, float* dL_dopacities,
                                    float* dL_dvelocities, float* dL_dsensors, void* stream) {
    splat_status st = check_gaussians(g, false);
    if (st != SPLAT_OK) return st;
    Frame fr;
    if ((st = build_frame(n_sensors, sensors, fr, nullptr)) != SPLAT_OK) return st;
    if ((st = check_proj(proj)) != SPLAT_OK) return st;
    if (!grad_proj || !dL_dmeans || !dL_dscales || !dL_dquats || !dL_dopacities)
        return fail(SPLAT_ERR_INVALID_ARG, "gradient pointer is NULL");
    if (!aligned16(grad_proj)) return fail(SPLAT_ERR_INVALID_ARG, "grad_proj misaligned");
    launch_project_backward(gauss_in(g), fr, proj.n_tiles, (const float4*)grad_proj,
                            GradOut{dL_dmeans, dL_dscales, dL_dquats, dL_dopacities, dL_dvelocities, dL_dsensors},
                            (cudaStream_t)stream);
    return check_launch("splat_project_backward");
}

splat_status splat_l1_loss(const float* pred, const float* target, int64_t count, float scale, float* grad,
                           float* loss, void* stream) {
    if (count < 0 || (count > 0 && (!pred || !target))) return fail(SPLAT_ERR_INVALID_ARG, "bad L1 arguments");
    launch_l1(pred, target, count, scale, grad, loss, (cudaStream_t)stream);
    return check_launch("splat_l1_loss");
}

int32_t splat_head_param_count(void) { return head_param_count(); }

splat_status splat_head_inputs(const splat_sensor* lidar, const float* feat, int32_t channels, float* x,
                               void* stream) {
    Frame fr;
    splat_status st = build_frame(1, lidar, fr, nullptr);
    if (st != SPLAT_OK) return st;
    if (fr.s[0].kind != SPLAT_SENSOR_LIDAR) return fail(SPLAT_ERR_INVALID_ARG, "splat_head_inputs needs a lidar");
    if (channels + 3 != 32) return fail(SPLAT_ERR_INVALID_ARG, "head input is 32 wide: channels must be 29");
    if (!feat || !x || !aligned16(x)) return fail(SPLAT_ERR_INVALID_ARG, "bad feature or input pointer");
    launch_head_inputs(fr.s[0], feat, channels, x, (cudaStream_t)stream);
    return check_launch("splat_head_inputs");
}

static splat_status check_head(const float* x, int64_t R, const uint16_t* w, const float* b) {
    if (R < 0) return fail(SPLAT_ERR_INVALID_ARG, "R < 0");
    if (R > 0 && (!x || !w || !b)) return fail(SPLAT_ERR_INVALID_ARG, "head pointer is NULL");
    if (!aligned16(x)) return fail(SPLAT_ERR_INVALID_ARG, "head inputs must be 16-byte aligned");
    return SPLAT_OK;
}

splat_status splat_head_forward(const float* x, int64_t R, const uint16_t* w_bf16, const float* bias, float* out,
                                void* stream) {
    splat_status st = check_head(x, R, w_bf16, bias);
    if (st != SPLAT_OK) return st;
    if (R > 0 && (!out || ((uintptr_t)out & 7u))) return fail(SPLAT_ERR_INVALID_ARG, "bad output pointer");
    launch_head_fwd(x, R, HeadW{w_bf16, bias}, out, (cudaStream_t)stream);
    return check_launch("splat_head_forward");
}

splat_status splat_head_train(const float* x, int64_t R, const uint16_t* w_bf16, const float* bias,
                              const float* y_int, const float* y_drop, float lam_i, float lam_d, float* grad,
                              float* loss, float* dx, void* stream) {
    splat_status st = check_head(x, R, w_bf16, bias);
    if (st != SPLAT_OK) return st;
    if (R > 0 && (!y_int || !y_drop || !grad)) return fail(SPLAT_ERR_INVALID_ARG, "bad target or gradient pointer");
    launch_head_train(x, R, HeadW{w_bf16, bias}, y_int, y_drop, lam_i, lam_d, grad, loss, dx, (cudaStream_t)stream);
    return check_launch("splat_head_train");
}

splat_status splat_head_adam(float* params, const float* grad, float* m, float* v, float lr, float beta1, float beta2,
                             float eps, int64_t step, uint16_t* w_bf16, float* bias, void* stream) {
    if (!params || !grad || !m || !v || !w_bf16 || !bias || step < 1)
        return fail(SPLAT_ERR_INVALID_ARG, "bad Adam arguments");
    launch_head_adam(params, grad, m, v, lr, beta1, beta2, eps, step, w_bf16, bias, (cudaStream_t)stream);
    return check_launch("splat_head_adam");
}

const char* splat_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace splat {
// Per-sensor constants of sensor `which` within a frame (its tile numbering included).
splat_status frame_sensor_constants(int32_t n_sensors, const splat_sensor* sensors, int32_t which, SensorDev* out) {
    Frame fr;
    const splat_status st = build_frame(n_sensors, sensors, fr, nullptr);
    if (st != SPLAT_OK) return st;
    if (which < 0 || which >= n_sensors) return fail(SPLAT_ERR_INVALID_ARG, "sensor index out of range");
    *out = fr.s[which];
    return SPLAT_OK;
}

// Status words of the translation units that raise them (status.cuh).
static StatusReader*& status_head() {
    static StatusReader* head = nullptr;
    return head;
}
void register_status_reader(StatusReader* r) {
    r->next = status_head();
    status_head() = r;
}
void take_all_status(uint32_t* bits, uint32_t* site) {
    for (StatusReader* r = status_head(); r; r = r->next) r->take(bits, site);
}

// Lets other translation units of the library report an error through splat_last_error().
splat_status record_error(splat_status code, const char* msg) {
    g_err = msg;
    return code;
}
}  // namespace splat
