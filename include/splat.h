/*
 * splat.h -- C ABI of libsplat, a GB300 (sm_103a) implementation of SplatAD's
 * differentiable tile-based Gaussian rasterizer for cameras and spinning lidars
 * (arXiv 2411.16816).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Every array argument is CALLER-OWNED DEVICE MEMORY unless stated otherwise; the
 *    library never allocates, frees or synchronises.  All work is enqueued on `stream`
 *    (a cudaStream_t passed as void*; NULL means the legacy default stream).
 *  - All floating point is FP32.  Matrices are row-major.
 *  - Host-detectable argument errors (null pointers, unsupported channel counts,
 *    inconsistent tiling) return SPLAT_ERR_INVALID_ARG before anything is enqueued;
 *    splat_last_error() then returns a message (thread-local).
 *  - Errors found on the device (intersection capacity exceeded) are reported through
 *    device-side counters described per function; nothing writes out of bounds.  In the
 *    checked build (libsplat_checked.so) every kernel also checks its indices against
 *    their buffers; a failing check skips the access and raises a device status word
 *    that splat_sync_status reports (SPLAT_ERR_BOUNDS).
 *  - Gradient outputs are ACCUMULATED (+=) so that several sensors or frames can share
 *    them; the caller zeroes them first.
 *  - The library launches no kernel that waits on another block: there are no
 *    inter-block spin waits anywhere, so no call can hang on a lost signal.  The one
 *    kernel that waits at all, the decoder's training pass on the tensor cores, waits only
 *    for its own block's matrix products, with a bound: if it runs out the block stops,
 *    and splat_sync_status returns SPLAT_ERR_TIMEOUT.
 *
 * Sensor model (paper Sec. 3.2, 3.3, App. A, App. D)
 * --------------------------------------------------
 *  World frame: any right-handed frame.  A sensor pose is the world->sensor rotation R
 *  and translation t (x_s = R x_w + t) at the sensor's mid-capture time; lin_vel and
 *  ang_vel are the sensor's own linear and angular velocity in its own frame.  Camera
 *  frame: z forward, x right, y down; pixel centres at (col + 0.5, row + 0.5).  Lidar
 *  frame: azimuth phi = atan2(y, x) in [0, 2 pi), elevation omega = asin(z / r).
 */
#ifndef SPLAT_H
#define SPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t splat_status;
#define SPLAT_OK 0
#define SPLAT_ERR_INVALID_ARG 1
#define SPLAT_ERR_CAPACITY 2
#define SPLAT_ERR_CUDA 3
#define SPLAT_ERR_TIMEOUT 4
#define SPLAT_ERR_BOUNDS 5

#define SPLAT_SENSOR_CAMERA 0
#define SPLAT_SENSOR_LIDAR 1
#define SPLAT_MAX_SENSORS 16

/* 3D Gaussians (paper Sec. 3.1), structure of arrays, device memory, FP32.
 *   means[n][3]       world-frame means mu
 *   scales[n][3]      ACTIVATED scales S (already exponentiated, > 0)
 *   quats[n][4]       rotation quaternion (w, x, y, z), need not be normalised
 *   opacities[n]      ACTIVATED opacity o in (0, 1)
 *   features[n][channels]  per-Gaussian features blended by the rasterizer (the
 *                     paper's [f_rgb, f]); channels in {1,2,3,4,8,16,29,32}
 *   velocities[n][3]  world-frame velocity of each Gaussian (v_dyn before rotation to
 *                     the sensor frame); may be NULL for a static scene */
typedef struct {
    const float *means;
    const float *scales;
    const float *quats;
    const float *opacities;
    const float *features;
    const float *velocities;
    int64_t n;
    int32_t channels;
    int32_t reserved;
} splat_gaussians;

/* One sensor.  `kind` selects which block of fields is read.
 * Camera (Sec. 3.2): pinhole width x height, fx, fy, cx, cy; rs_time is the rolling-
 *   shutter readout time t_rs (first to last row, seconds; 0 = global shutter);
 *   time_offset is the learnable offset between timestamp and mid-exposure (added to
 *   every row time); eps2d is the blur s of Eq. (alpha) in px^2 (0.3 in the paper);
 *   near_plane culls Gaussians with camera z below it; tile_w x tile_h is the tile
 *   (16 x 16 in the paper; supported: 16x16, 8x8, 32x8, 16x32).
 * Lidar (Sec. 3.3, App. A): n_beams elevation channels with ascending elevations
 *   beam_elev[n_beams] (radians, DEVICE memory), n_az azimuth bins of az_res radians
 *   (n_az * az_res must equal 2 pi), sweep_time is the spin period t_rs, eps2d is the
 *   blur in rad^2, r_min culls Gaussians closer than it (metres); tile_w x tile_h =
 *   N_phi azimuth bins x N_omega beams per tile (32 x 8 in the paper; n_beams must be
 *   a multiple of tile_h and tile_w * tile_h must be 64, 128, 256 or 512).  rays, if
 *   not NULL, is DEVICE memory [n_beams][n_az][3] of per-ray (phi, omega, t) that
 *   replace the regular grid phi = (a + 0.5) az_res, omega = beam_elev[b],
 *   t = ((a + 0.5) / n_az - 0.5) sweep_time; each ray stays in its grid cell's tile. */
typedef struct {
    int32_t kind;
    int32_t reserved0;
    float R[9];
    float t[3];
    float lin_vel[3];
    float ang_vel[3];
    /* camera */
    int32_t width, height;
    float fx, fy, cx, cy;
    float rs_time, time_offset;
    float eps2d;
    float near_plane;
    /* lidar */
    int32_t n_beams, n_az;
    const float *beam_elev;
    const float *rays;
    float az_res, sweep_time, r_min;
    /* tiling (both kinds) */
    int32_t tile_w, tile_h;
    /* tile extent of a Gaussian, flags (0: the paper's box of 3 standard deviations of
     * Sigma' plus the motion margin |v| t_rs / 2, Sec. 3.2, Sec. 3.3):
     *   1  opacity-aware: sqrt(2 ln(255 o')) standard deviations -- exactly the bounding
     *      box of the ellipse where alpha can reach 1/255, so the tile lists then hold
     *      every Gaussian a ray of the tile can blend;
     *   2  lidar only, regular ray grid only (rays == NULL): the motion margins use the
     *      fire times of the grid rays, t(phi) = phi t_sweep / (n_az az_res) - t_sweep / 2,
     *      instead of the whole sweep (a box crossing azimuth 0 keeps the full margins);
     *      such a lidar's lists then serve its grid rays only, and the free-ray entry
     *      points reject it;
     *   4  camera tile cull (no effect on a lidar): a tile of the box is listed only if
     *      the Gaussian can reach alpha >= 1/255 at one of its pixels at that pixel's row
     *      time -- if its rectangle of pixel centres, grown per axis by the mean's motion
     *      over half the tile's row-time span and by 2e-3 px, meets the ellipse
     *      d^T Sigma'^-1 d <= 2 ln(255 o') (1 + 2e-3) + 2e-3.  The margins keep every pair
     *      an FP32 alpha test could blend, so renders and gradients are those of the
     *      uncut lists; the lists (and the sort, and the raster's staging) shrink by the
     *      pairs that blend nowhere in their tile (about a third on driving scenes). */
    int32_t support;
} splat_sensor;

/* Per-(sensor, Gaussian) projection results, caller-owned device buffers.
 *   rec[n_sensors][3][n][4] floats:
 *     rec[s][0][i] = (mean_a, mean_b, v_a, v_b)  2-D mean (pixels, or phi/omega in rad)
 *                     and its sensor-space velocity (Eq. pixel velocity / v^S)
 *     rec[s][1][i] = (conic_a, conic_b, conic_c, o')  (Sigma_2d + eps I)^-1 as
 *                     [[a, b], [b, c]] and the compensated opacity of Eq. (alpha)
 *     rec[s][2][i] = (depth, v_r, 0, 0)  camera z or lidar range r, and the range rate
 *   rect[n_sensors][n][4] int16: tile rectangle (x0, y0, x1, y1), x1/y1 exclusive; for
 *     a lidar x0 is in [0, M_phi) and x1 may exceed M_phi (columns wrap modulo M_phi)
 *   n_tiles[n_sensors][n] int32: intersected tiles (0 = culled) */
typedef struct {
    float *rec;
    int16_t *rect;
    int32_t *n_tiles;
} splat_projected;

/* Sorted intersection lists of a frame (all sensors).
 *   isect_ids[capacity]: Gaussian index of each (tile, Gaussian) pair, ordered by
 *     global tile, then depth (camera z / lidar range), then Gaussian index.
 *   tile_ranges[total_tiles][2]: [start, end) of each tile in isect_ids.  Global tile
 *     ids number the sensors' tiles consecutively in sensor order, each sensor
 *     row-major (camera: ty * tiles_x + tx; lidar: row * M_phi + column).
 *   n_isect: one int64 on the device, written with the number of intersections found
 *     (it may exceed `capacity`, in which case the lists are not valid). */
typedef struct {
    uint32_t *isect_ids;
    int32_t *tile_ranges;
    int64_t *n_isect;
} splat_bins;

/* Tiles of a frame: per-sensor tile counts, their total, and rays per sensor.
 * tiles_out and rays_out are HOST arrays of n_sensors entries (may be NULL). */
splat_status splat_frame_layout(int32_t n_sensors, const splat_sensor *sensors, int64_t *total_tiles,
                                int64_t *tiles_out, int64_t *rays_out);

/* Bytes of device workspace splat_bin_sort needs for n Gaussians, the given sensors and
 * an intersection capacity. */
splat_status splat_workspace_size(int64_t n, int32_t n_sensors, const splat_sensor *sensors, int64_t capacity,
                                  size_t *bytes);

/* Projection of every Gaussian into every sensor (Sec. 3.2 "Projection, tiling, and
 * sorting", Eq. pixel velocity, App. D; Sec. 3.3 Eq. spherical projection, J^S, v^S,
 * App. A.1 tile ranges).  Writes proj.rec (visible Gaussians only), proj.rect and
 * proj.n_tiles for all n_sensors x n pairs. */
splat_status splat_project(const splat_gaussians *g, int32_t n_sensors, const splat_sensor *sensors,
                           splat_projected proj, void *stream);

/* Input health (no counterpart in the paper).  splat_project culls from every sensor a
 * Gaussian whose mean, scale, quaternion, opacity or velocity holds a NaN or an infinity
 * (and one whose quaternion is zero): it takes no tile, is never blended and receives no
 * gradient.  This call adds to *count (one device int64, accumulated) the number of
 * Gaussians with such a non-finite parameter; features are not inspected (a non-finite
 * feature reaches the outputs of the rays that blend it).  Asynchronous; g's features
 * may be NULL. */
splat_status splat_count_nonfinite(const splat_gaussians *g, int64_t *count, void *stream);

/* Tile duplication and sort (Sec. 3.2 tiling and depth sort; Sec. 3.3 range sort;
 * App. A.1 wrapped identifiers).  Emits every (tile, Gaussian) pair of the frame,
 * orders them by (tile, depth, Gaussian index) with an on-device stable radix sort and
 * writes per-tile ranges.  `workspace` is device scratch of at least
 * splat_workspace_size() bytes.  If more than `capacity` pairs exist, *bins.n_isect
 * holds the required count, the lists are left undefined, and the call returns
 * SPLAT_OK (the caller checks n_isect against capacity, grows its buffers and calls
 * again).  The sort's row items (the tile rows of the visible boxes) share the
 * capacity: when they alone exceed it, n_isect reports their number (the capacity
 * needed) in the same way. */
splat_status splat_bin_sort(int64_t n, int32_t n_sensors, const splat_sensor *sensors, splat_projected proj,
                            int64_t capacity, splat_bins bins, void *workspace, size_t workspace_bytes,
                            void *stream);

/* splat_bin_sort for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a deployment convenience).  Hosts with a fixed device-memory
 * budget, plug-ins running inside another program's frame loop, or runtimes that forbid
 * allocation after start-up cannot hand the sort a workspace; this variant takes its
 * scratch from a 32 MiB array built into the library (held by every GPU that loads the
 * library until the process exits), so it allocates nothing.  Arguments and results are
 * those of splat_bin_sort without the workspace.  A frame whose scratch need
 * (splat_workspace_size) exceeds 32 MiB is rejected with SPLAT_ERR_INVALID_ARG before
 * anything is enqueued.  The first call on a device looks up the array's device address
 * and keeps it for the device's current CUDA context; make that call before any stream
 * capture.  After cudaDeviceReset the next call sees a new context and looks the address
 * up again (again outside any capture).  A call that needs the look-up while its stream
 * is capturing returns SPLAT_ERR_INVALID_ARG and enqueues nothing.  All calls share the
 * array, so calls whose work overlaps on the GPU race; nothing in it needs to start at
 * zero. */
splat_status splat_bin_sort_noalloc(int64_t n, int32_t n_sensors, const splat_sensor *sensors, splat_projected proj,
                                    int64_t capacity, splat_bins bins, void *stream);

/* The sort has no gradient: this twin exists for symmetry and does nothing. */
splat_status splat_bin_sort_backward(void);

/* Camera rasterization (Eq. t_pix, alpha blend, alpha, delta) of every camera sensor in
 * the frame, one CTA per tile.  Outputs are concatenated over the frame's cameras in
 * sensor order, each row-major H x W:
 *   out_feat[pixels][channels]  blended features
 *   out_T[pixels]               final transmittance
 *   out_last[pixels]            number of list entries up to and including the last
 *                               Gaussian blended into the pixel (for the backward pass);
 *                               out_T and out_last may be NULL.
 *   evaluated                   optional device uint64 to which the number of (pixel,
 *                               Gaussian) pairs examined is added (work accounting). */
splat_status splat_render_camera(const splat_gaussians *g, int32_t n_sensors, const splat_sensor *sensors,
                                 splat_projected proj, splat_bins bins, float *out_feat, float *out_T,
                                 int32_t *out_last, uint64_t *evaluated, void *stream);

/* Camera rasterization with the L1 photometric term (Eq. loss_fn, lambda_r L1) fused into
 * its epilogue: the same render as splat_render_camera, then, per ray and channel,
 * loss += scale * |F - target| and grad_feat = scale * sign(F - target) (the upstream
 * gradient of splat_render_camera_backward), without a separate pass over the images.
 *   target[rays][C]     device, the reference image(s) in out_feat's layout; 16-byte
 *                       aligned when C % 4 == 0 (so are grad_feat and out_feat)
 *   grad_feat[rays][C]  device, written (not accumulated)
 *   loss                device float, accumulated (the caller zeroes it)
 *   out_feat            may be NULL when the rendered image itself is not wanted;
 *                       out_T, out_last and evaluated as for splat_render_camera. */
splat_status splat_render_camera_l1(const splat_gaussians *g, int32_t n_sensors, const splat_sensor *sensors,
                                    splat_projected proj, splat_bins bins, const float *target, float scale,
                                    float *out_feat, float *out_T, int32_t *out_last, float *grad_feat,
                                    float *loss, uint64_t *evaluated, void *stream);

/* Lidar rasterization (Sec. 3.3: blended features, expected range of the rolling-
 * shutter ranges r + v_r t, median range = rolling-shutter range of the first Gaussian
 * after which the transmittance is below 0.5, 0 if none).  Outputs are concatenated
 * over the frame's lidars in sensor order, each [n_beams][n_az]:
 *   out_feat[rays][channels], out_range_exp[rays], out_range_med[rays],
 *   out_alpha[rays] (= 1 - T), out_T[rays], out_last[rays] (as for cameras);
 *   out_range_med, out_T and out_last may be NULL; evaluated as for cameras. */
splat_status splat_render_lidar(const splat_gaussians *g, int32_t n_sensors, const splat_sensor *sensors,
                                splat_projected proj, splat_bins bins, float *out_feat, float *out_range_exp,
                                float *out_range_med, float *out_alpha, float *out_T, int32_t *out_last,
                                uint64_t *evaluated, void *stream);

/* Line-of-sight term of the training loss (App. B, lambda_los L_los): for a lidar ray p
 * with a measured return at range r_p, L_los,p = sum of alpha_i over the Gaussians the
 * ray blends whose rolling-shutter range r_rs,i = r_i + v_r,i t_p lies before
 * r_p - eps.  The term rides on the lidar traversal.
 *   target_range[lidar rays]  device, in out_feat's ray order; <= 0 marks a ray without
 *                             a return (its term is 0)
 *   eps                       metres (the paper uses 0.8), >= 0 */
typedef struct {
    const float *target_range;
    float eps;
    int32_t reserved;
} splat_los;

/* splat_render_lidar plus the line-of-sight term of every lidar ray in out_los[rays]
 * (device, written).  The other outputs are exactly those of splat_render_lidar. */
splat_status splat_render_lidar_los(const splat_gaussians *g, int32_t n_sensors, const splat_sensor *sensors,
                                    splat_projected proj, splat_bins bins, float *out_feat, float *out_range_exp,
                                    float *out_range_med, float *out_alpha, float *out_T, int32_t *out_last,
                                    splat_los los, float *out_los, uint64_t *evaluated, void *stream);

/* Lidar rendering with the per-ray decoder fused into the raster epilogue (Sec. 3.3:
 * the rendered features and the ray direction are decoded per ray into intensity and
 * ray-drop; App. B: the two-hidden-layer decoder).  Renders every lidar sensor of the
 * frame exactly as splat_render_lidar does (out_feat may be NULL: the features are then
 * not written) and decodes each ray's 29 rendered channels and unit direction
 * (cos w cos phi, cos w sin phi, sin w) with the decoder's BF16 weights head_w (W1 | W2 |
 * W3, row-major [in][out], as splat_head_train keeps them) and FP32 biases head_b into
 * out_head[rays][2] = (intensity logit, ray-drop logit).  The result equals
 * splat_head_inputs followed by splat_head_forward bit for bit, without the rendered
 * features passing through device memory.  Requires channels == 29 and the lidar tile
 * 32 x 8 (else SPLAT_ERR_INVALID_ARG); out_head 8-byte aligned.  Asynchronous. */
splat_status splat_render_lidar_head(const splat_gaussians *g, int32_t n_sensors, const splat_sensor *sensors,
                                     splat_projected proj, splat_bins bins, float *out_feat, float *out_range_exp,
                                     float *out_range_med, float *out_alpha, float *out_T, int32_t *out_last,
                                     const uint16_t *head_w, const float *head_b, float *out_head, void *stream);

/* Backward of splat_render_camera.  Inputs: the forward's out_T and out_last (or both
 * NULL: the kernel then recomputes them per tile), dL_dfeat[pixels][channels] and
 * dL_dT[pixels] (may be NULL).  Accumulates into
 *   grad_proj[n_sensors][3][n][4]: gradients of proj.rec (same layout),
 *   dL_dfeatures[n][channels], and, if dL_dsensors is not NULL, entry 6 of
 *   dL_dsensors[n_sensors][16] of every camera: the gradient with respect to its time
 *   offset (the camera "time to centre" the paper optimises; every pixel time of Eq.
 *   t_pix carries it).
 * For 9-16 channels on 256-ray tiles the two channel contractions of the reverse mode
 * (the upstream gradient's dot products with the features, and dL_dfeatures) are formed
 * on the tensor cores from split BF16 operands (hi + lo) with FP32 accumulation, about
 * 2^-16 relative per term; everything else is FP32. */
splat_status splat_render_camera_backward(const splat_gaussians *g, int32_t n_sensors, const splat_sensor *sensors,
                                          splat_projected proj, splat_bins bins, const float *out_T,
                                          const int32_t *out_last, const float *dL_dfeat, const float *dL_dT,
                                          float *grad_proj, float *dL_dfeatures, float *dL_dsensors,
                                          void *stream);

/* Backward of splat_render_lidar for dL_dfeat[rays][channels], dL_drange_exp[rays] and
 * dL_dalpha[rays] (the latter two may be NULL).  The median range has no gradient.
 * out_T/out_last as for cameras (both NULL: recomputed).  Accumulates like the camera
 * twin. */
splat_status splat_render_lidar_backward(const splat_gaussians *g, int32_t n_sensors, const splat_sensor *sensors,
                                         splat_projected proj, splat_bins bins, const float *out_T,
                                         const int32_t *out_last, const float *dL_dfeat,
                                         const float *dL_drange_exp, const float *dL_dalpha, float *grad_proj,
                                         float *dL_dfeatures, void *stream);

/* splat_render_lidar_backward plus the gradient of sum_p dL_dlos[p] * L_los,p (the
 * line-of-sight term above, same los): each blended alpha_i in front of the cut gets
 * dL_dlos[p] added to its upstream gradient.  dL_dlos[lidar rays] is device memory. */
splat_status splat_render_lidar_backward_los(const splat_gaussians *g, int32_t n_sensors,
                                             const splat_sensor *sensors, splat_projected proj, splat_bins bins,
                                             const float *out_T, const int32_t *out_last, const float *dL_dfeat,
                                             const float *dL_drange_exp, const float *dL_dalpha, splat_los los,
                                             const float *dL_dlos, float *grad_proj, float *dL_dfeatures,
                                             void *stream);

/* ---- Lidar point clouds as rays (App. A.2) ------------------------------------------
 * A lidar's measured points arrive ego-motion compensated: in its sensor frame at the
 * sweep's reference time.  Rendering them needs the rays they were measured along:
 * splat_lidar_points_to_rays undoes the compensation with the sensor's constant linear
 * and angular velocity (lin_vel, ang_vel of splat_sensor, sensor frame), a static point
 * p captured at time t appearing at q = p - t (lin_vel + ang_vel x p), and takes q's
 * azimuth phi = atan2(q_y, q_x) in [0, 2 pi), elevation omega = asin(q_z / |q|) and t.
 * Each ray belongs to the tile a zero-extent Gaussian at (phi, omega) would: column
 * floor(phi / (tile_w az_res)) (the last column also takes the rest of the circle), the
 * tile row whose elevation boundaries (those of the lidar tiling, App. A.1) hold omega;
 * none (-1) outside the beam fan.  splat_lidar_bin_rays groups the rays by that tile
 * and splat_render_lidar_rays renders them against the frame's projection and sorted
 * lists, exactly as the grid rays of that tile are rendered (the rays' times should lie
 * within the sweep, [-sweep_time/2, sweep_time/2], which the tiles' motion margins
 * cover).  Rays outside every tile are not rendered and their outputs not written. */

/* One lidar's free rays grouped by tile (device memory, caller-owned).
 *   ray_ids[n_rays]       ray indices grouped by tile; the first tile_ranges[tiles-1][1]
 *                         entries are used, the order inside a tile is unspecified
 *   tile_ranges[tiles][2] (start, end) of each tile of the lidar in ray_ids
 *   chunk_base[tiles + 1] first 256-ray work chunk of each tile; [tiles] = the number of
 *                         chunks (sum over tiles of ceil(count / 256))
 * tiles = ceil(n_az / tile_w) * (n_beams / tile_h) of that lidar. */
typedef struct {
    int32_t *ray_ids;
    int32_t *tile_ranges;
    int32_t *chunk_base;
} splat_ray_bins;

/* points[n_points][3] (float, sensor frame at the reference time), times[n_points]
 * (seconds relative to it) -> rays[n_points][3] (phi, omega, t), ranges[n_points] (|q|,
 * the measured range along the ray) and, if tiles is not NULL, tiles[n_points] (the
 * lidar's local tile of each ray, -1 outside the fan).  `lidar` indexes a lidar sensor
 * of the table.  FP32; n_points < 2^31. */
splat_status splat_lidar_points_to_rays(int32_t n_sensors, const splat_sensor *sensors, int32_t lidar,
                                        const float *points, const float *times, int64_t n_points, float *rays,
                                        float *ranges, int32_t *tiles, void *stream);

/* Counting sort of rays[n_rays][3] (phi, omega, t; e.g. from splat_lidar_points_to_rays)
 * by their tile of lidar `lidar` into bins (written; see splat_ray_bins). */
splat_status splat_lidar_bin_rays(int32_t n_sensors, const splat_sensor *sensors, int32_t lidar, const float *rays,
                                  int64_t n_rays, splat_ray_bins bins, void *stream);

/* Training-time grouping (App. A.2: a tile may receive more rays than its 256 threads,
 * e.g. where the linear ego-motion model is violated; training shuffles each iteration
 * and drops the rays beyond 256).  Groups like splat_lidar_bin_rays, then each tile
 * keeps the `cap` rays (cap >= 1; 256 for one pass per tile) of smallest key
 * (priority[ray] << 32 | ray), listed in key order; the others are dropped (not
 * rendered, outputs not written).  priority[n_rays] (uint32, device) is the caller's
 * random draw -- fresh values each iteration shuffle which rays a full tile keeps.
 * `scratch` holds the uncapped grouping (same sizes as bins; caller-owned, overwritten). */
splat_status splat_lidar_bin_rays_capped(int32_t n_sensors, const splat_sensor *sensors, int32_t lidar,
                                         const float *rays, const uint32_t *priority, int64_t n_rays, int32_t cap,
                                         splat_ray_bins scratch, splat_ray_bins bins, void *stream);

/* Renders the binned rays of lidar `lidar` (sensor table as for the frame's projection
 * and bins).  Outputs are indexed by ray: out_feat[n_rays][channels], out_range_exp,
 * out_range_med, out_alpha, out_T, out_last [n_rays] with the meaning of
 * splat_render_lidar (out_range_med, out_T, out_last may be NULL).  los may be NULL;
 * otherwise its target_range is indexed by ray (e.g. the ranges of
 * splat_lidar_points_to_rays) and out_los[n_rays] receives the line-of-sight term. */
splat_status splat_render_lidar_rays(const splat_gaussians *g, int32_t n_sensors, const splat_sensor *sensors,
                                     int32_t lidar, splat_projected proj, splat_bins bins, const float *rays,
                                     int64_t n_rays, splat_ray_bins ray_bins, float *out_feat,
                                     float *out_range_exp, float *out_range_med, float *out_alpha, float *out_T,
                                     int32_t *out_last, const splat_los *los, float *out_los, void *stream);

/* Backward of splat_render_lidar_rays: upstream gradients indexed by ray as its outputs
 * (dL_drange_exp, dL_dalpha may be NULL; dL_dlos only with los, else NULL), out_T and
 * out_last of the forward or both NULL (recomputed).  Accumulates into grad_proj and
 * dL_dfeatures like splat_render_lidar_backward.  The rays are data: no gradient flows
 * into the points or the sensor through them. */
splat_status splat_render_lidar_rays_backward(const splat_gaussians *g, int32_t n_sensors,
                                              const splat_sensor *sensors, int32_t lidar, splat_projected proj,
                                              splat_bins bins, const float *rays, int64_t n_rays,
                                              splat_ray_bins ray_bins, const float *out_T, const int32_t *out_last,
                                              const float *dL_dfeat, const float *dL_drange_exp,
                                              const float *dL_dalpha, const splat_los *los, const float *dL_dlos,
                                              float *grad_proj, float *dL_dfeatures, void *stream);

/* Chain rule from grad_proj to the Gaussian parameters, summed over sensors (one thread
 * per Gaussian, no atomics).  Accumulates into dL_dmeans[n][3], dL_dscales[n][3],
 * dL_dquats[n][4], dL_dopacities[n], dL_dvelocities[n][3] (may be NULL).  Gradients
 * are with respect to the ACTIVATED scales and opacities and the unnormalised
 * quaternion.  If dL_dsensors is not NULL, dL_dsensors[n_sensors][16] accumulates, per
 * sensor and summed over the Gaussians (one atomic per warp): entries 0..2 and 3..5, the
 * gradients with respect to its linear and angular velocity (sensor frame, through the
 * relative velocity of Eq. pixel velocity / App. D; the paper optimises both); 8..10,
 * its translation t (mu_sensor = R mu + t); 11..13, its rotation, perturbed as
 * R <- (I + [theta]x) R with theta in the sensor frame.  Entry 6 is the camera time
 * offset (splat_render_camera_backward); 7, 14, 15 are unused. */
splat_status splat_project_backward(const splat_gaussians *g, int32_t n_sensors, const splat_sensor *sensors,
                                    splat_projected proj, const float *grad_proj, float *dL_dmeans,
                                    float *dL_dscales, float *dL_dquats, float *dL_dopacities,
                                    float *dL_dvelocities, float *dL_dsensors, void *stream);

/* L1 term of the training loss (Eq. loss_fn, lambda_r L1): adds scale * sum |pred - target|
 * over `count` floats to *loss (device float, accumulated) and, if grad is not NULL,
 * writes grad[i] = scale * sign(pred[i] - target[i]).  loss may be NULL. */
splat_status splat_l1_loss(const float *pred, const float *target, int64_t count, float scale, float *grad,
                           float *loss, void *stream);

/* ---------------------------------------------------------------------------------
 * Batched rendering: many camera views and lidar sweeps of different sizes, over several
 * scenes, rasterized by ONE persistent launch (forward only, for serving).  The paper
 * renders one sensor at a time; this is the serving form of its rasterization
 * (Sec. 3.2, 3.3).
 *
 * Each request names a sensor that was projected and binned as part of a group (a frame
 * passed to splat_project / splat_bin_sort), the group's buffers, its scene's features
 * and its own outputs (layouts as for splat_render_camera / splat_render_lidar of a single
 * sensor).  Every request's tile must hold 256 rays (tile_w * tile_h == 256).
 * --------------------------------------------------------------------------------- */
typedef struct {
    const splat_sensor *group_sensors;  /* HOST array: the group's sensors, as binned */
    int32_t group_n_sensors;
    int32_t group_sensor_index;         /* this request's sensor within the group */
    splat_projected proj;               /* the group's projection buffers */
    splat_bins bins;                    /* the group's sorted lists */
    const float *features;              /* the scene's features [n][channels] */
    int64_t n;
    int32_t channels;
    int32_t reserved;
    float *out_feat;                    /* [rays][channels] */
    float *out_T;                       /* [rays] or NULL */
    float *out_range_exp;               /* lidar: [rays] */
    float *out_range_med;               /* lidar: [rays] or NULL */
    float *out_alpha;                   /* lidar: [rays] */
} splat_batch_request;

/* Bytes of the request table for n requests (1..1024). */
size_t splat_batch_table_bytes(int32_t n_requests);

/* Writes the request table into `table` (HOST memory of splat_batch_table_bytes bytes)
 * and the number of work items (tiles over all requests) into *total_items.  The caller
 * copies the table to device memory once; it stays valid while the buffers it names do.
 * Requests are processed in table order (put the largest first for throughput). */
splat_status splat_batch_build(const splat_batch_request *reqs, int32_t n_requests, void *table, size_t table_bytes,
                               int64_t *total_items);

/* Renders every request of a DEVICE copy of the table in one persistent launch.
 * counters: device int32[n_requests + 1] (reset by this call); stamps, if not NULL:
 * device uint64[n_requests + 1] receiving the global-timer nanoseconds at which each
 * request's last tile finished, and in stamps[n_requests] the time the batch started.
 * max_channels is the largest channel count of the requests (<= 32).  evaluated, if not
 * NULL: device uint64[2] to which the (ray, Gaussian) pairs the launch examines are
 * added (cameras, lidars) -- a counting variant of the kernel, for work accounting.
 * Safe to capture in a CUDA graph (it enqueues a memset and two kernels). */
splat_status splat_render_batch(const void *table, int32_t n_requests, int64_t total_items, int32_t max_channels,
                                int32_t *counters, uint64_t *stamps, uint64_t *evaluated, void *stream);

/* Writes the device global timer (nanoseconds) to the device uint64 *at when the stream
 * reaches this point (latency bookkeeping for batches). */
splat_status splat_stamp(uint64_t *at, void *stream);

/* ---------------------------------------------------------------------------------
 * Per-ray lidar decoder (paper Sec. 3.3: the rendered features concatenated with the
 * ray direction are decoded to intensity and ray-drop probability by a small MLP;
 * App. B: two hidden layers, loss weights lambda_intens = 1 and lambda_raydrop = 0.1).
 * Network: x[32] -> relu(64) -> relu(64) -> (intensity logit, drop logit).
 * Parameters, flattened in this order (splat_head_param_count() = 6402 values):
 *   W1[32][64], b1[64], W2[64][64], b2[64], W3[64][2], b3[2]   (row-major [in][out]).
 * The decoder reads BF16 weights w_bf16 = W1 | W2 | W3 (6272 values) and FP32 biases
 * bias = b1 | b2 | b3 (130 values); products are accumulated in FP32 with FP32
 * activations.  All arrays are device memory.
 * --------------------------------------------------------------------------------- */
int32_t splat_head_param_count(void);

/* x[r] = [feat[r][0..channels), unit ray direction (cos w cos p, cos w sin p, sin w)] for
 * every ray of one lidar ([n_beams][n_az] order, grid or explicit rays); channels must be
 * 29 so that x is 32 wide.  x must be 16-byte aligned. */
splat_status splat_head_inputs(const splat_sensor *lidar, const float *feat, int32_t channels, float *x,
                               void *stream);

/* out[r] = (intensity logit, drop logit) for R rays; intensity = sigmoid(out[r][0]) and the
 * ray-drop probability = sigmoid(out[r][1]). */
splat_status splat_head_forward(const float *x, int64_t R, const uint16_t *w_bf16, const float *bias, float *out,
                                void *stream);

/* Training pass over R rays: loss = lam_i mean (sigmoid(o0) - y_int)^2 + lam_d mean
 * BCE(o1, y_drop), added to *loss (device float; may be NULL); its gradients with respect to
 * the 6402 parameters are ADDED to grad (FP32, caller zeroes); dx[R][32], if not NULL,
 * receives dL/dx (to continue the backward into the rasterizer's features). */
splat_status splat_head_train(const float *x, int64_t R, const uint16_t *w_bf16, const float *bias,
                              const float *y_int, const float *y_drop, float lam_i, float lam_d, float *grad,
                              float *loss, float *dx, void *stream);

/* One Adam step (bias-corrected, epsilon outside the square root) on the FP32 master
 * parameters `params` (6402 values) with moments m, v; then refreshes the decoder's BF16
 * weights (round to nearest even) and FP32 biases.  step counts from 1. */
splat_status splat_head_adam(float *params, const float *grad, float *m, float *v, float lr, float beta1,
                             float beta2, float eps, int64_t step, uint16_t *w_bf16, float *bias, void *stream);

/* Message of the last non-OK status on this host thread ("" if none). */
const char *splat_last_error(void);

/* Waits for the stream and reports a CUDA error raised by anything enqueued on it as
 * SPLAT_ERR_CUDA (message in splat_last_error).  It then reads and clears the device
 * status words of the current device: SPLAT_ERR_TIMEOUT if a bounded wait for tensor-core
 * work ran out, SPLAT_ERR_BOUNDS if the checked build skipped an out-of-bounds index, since
 * the last call (the message names the first site).  Capacity
 * overflow is not a status: it is reported through bins.n_isect.  Synchronous. */
splat_status splat_sync_status(void *stream);

/* 1 if this library is the checked build (every kernel index checked against its
 * buffer; a failing check skips the access and raises SPLAT_ERR_BOUNDS), else 0. */
int32_t splat_build_flags(void);

#ifdef __cplusplus
}
#endif
#endif /* SPLAT_H */
