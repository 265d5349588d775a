// common.cuh -- device-side frame descriptor and small math shared by the kernels of
// libsplat.  Everything here is FP32; constants follow the 3DGS conventions the paper
// builds on (alpha threshold 1/255, alpha clamp 0.999, early stop below T = 1e-4).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/splat.h"

namespace splat {

constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.999f;
constexpr float kTEps = 1e-4f;
constexpr float kTwoPi = 6.283185307179586f;
constexpr float kPi = 3.14159265358979f;
constexpr int kMaxSensors = SPLAT_MAX_SENSORS;

// Per-sensor constants, derived once on the host and passed by value in kernel params.
struct SensorDev {
    int kind;
    int tiles_x, tiles_y;
    int tile_w, tile_h;
    int tile_base;   // first global tile id of this sensor
    int block_base;  // first block of this sensor in its kind's raster launch
    int ray_base;    // first output ray (pixel) of this sensor in its kind's outputs
    int support;     // tile extent flags: 1 opacity-aware, 2 lidar margins from the rays' fire times,
                     // 4 camera tile cull
    float R[9], t[3], v[3], w[3];
    // camera
    int width, height;
    float fx, fy, cx, cy, rs, dt, eps, near_plane, lim_x, lim_y;
    // lidar
    int nb, naz;
    const float* elev;
    const float* rays;
    float az_res, sweep, rmin, wphi, phimax;
};

struct Frame {
    int n_sensors;
    int n_cam_blocks, n_lid_blocks;
    int cam_sensors[kMaxSensors];  // sensor indices of the cameras, in order
    int lid_sensors[kMaxSensors];
    int n_cams, n_lids;
    SensorDev s[kMaxSensors];
};

// The frame table travels by value in every launch; keep it inside the classic 4 KB
// kernel-parameter space together with the other arguments.
static_assert(sizeof(Frame) + 512 <= 4096, "frame table too large for kernel parameters");

// Projected record and gradient layout: [sensor][3][n] float4.
__host__ __device__ inline size_t rec_index(int s, int k, int64_t n, int64_t i) {
    return ((size_t)s * 3 + k) * (size_t)n + (size_t)i;
}

struct Mat3 {
    float m[9];
};

__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float* R) {
    R[0] = 1.f - 2.f * (y * y + z * z);
    R[1] = 2.f * (x * y - w * z);
    R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);
    R[4] = 1.f - 2.f * (x * x + z * z);
    R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);
    R[7] = 2.f * (y * z + w * x);
    R[8] = 1.f - 2.f * (x * x + y * y);
}

// Symmetric 3x3 stored as (xx, xy, xz, yy, yz, zz).
struct Sym3 {
    float xx, xy, xz, yy, yz, zz;
};

// R S R^T for symmetric S.
__device__ __forceinline__ Sym3 rotate_sym(const float* R, const Sym3& S) {
    // T = R S (3x3)
    float T[9];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        float r0 = R[3 * i], r1 = R[3 * i + 1], r2 = R[3 * i + 2];
        T[3 * i + 0] = r0 * S.xx + r1 * S.xy + r2 * S.xz;
        T[3 * i + 1] = r0 * S.xy + r1 * S.yy + r2 * S.yz;
        T[3 * i + 2] = r0 * S.xz + r1 * S.yz + r2 * S.zz;
    }
    Sym3 o;
    o.xx = T[0] * R[0] + T[1] * R[1] + T[2] * R[2];
    o.xy = T[0] * R[3] + T[1] * R[4] + T[2] * R[5];
    o.xz = T[0] * R[6] + T[1] * R[7] + T[2] * R[8];
    o.yy = T[3] * R[3] + T[4] * R[4] + T[5] * R[5];
    o.yz = T[3] * R[6] + T[4] * R[7] + T[5] * R[8];
    o.zz = T[6] * R[6] + T[7] * R[7] + T[8] * R[8];
    return o;
}

__device__ __forceinline__ float sym_get(const Sym3& S, int i, int j) {
    const int a = i < j ? i : j, b = i < j ? j : i;
    if (a == 0) return b == 0 ? S.xx : (b == 1 ? S.xy : S.xz);
    if (a == 1) return b == 1 ? S.yy : S.yz;
    return S.zz;
}

// Azimuth difference wrapped to [-pi, pi).
__device__ __forceinline__ float wrap_pi(float d) {
    return d - kTwoPi * floorf(d * (1.0f / kTwoPi) + 0.5f);
}

// Elevation boundary k of the lidar's tile rows (App. A.1): below the first beam by half
// its spacing, midway between the last beam of a row and the first of the next, above
// the last beam by half its spacing.
__device__ __forceinline__ float elev_bound(const SensorDev& S, int k) {
    const int Mw = S.nb / S.tile_h;
    const float* e = S.elev;
    if (k == 0) return e[0] - 0.5f * (e[1] - e[0]);
    if (k >= Mw) return e[S.nb - 1] + 0.5f * (e[S.nb - 1] - e[S.nb - 2]);
    return 0.5f * (e[k * S.tile_h - 1] + e[k * S.tile_h]);
}

// Half-extent of a Gaussian's tile box in standard deviations of Sigma': the paper's 3,
// or (opacity-aware) the radius of the ellipse where o' exp(-d^T Sigma'^-1 d / 2) can
// still reach 1/255, d^T Sigma'^-1 d <= 2 ln(255 o').
__device__ __forceinline__ float support_sigmas(const SensorDev& S, float op) {
    return (S.support & 1) ? sqrtf(fmaxf(2.f * logf(255.f * op), 0.f)) : 3.f;
}

// Camera tile cull (support flag 4).  A pixel of a tile row at its time t (Eq. t_pix) sees
// the mean at mean + v t (Eq. delta), i.e. acts as a point within |v| (t1 - t0) / 2 per
// axis of the pixel-centre rectangle around the mean at the row's mid-time.  A tile is
// kept when its rectangle, grown by that sweep and by 2e-3 px, meets the ellipse
// d^T K d <= 2 ln(255 o') (1 + 2e-3) + 2e-3 where alpha (Eq. alpha) could reach 1/255
// (the margins keep every pair an FP32 alpha could blend): the tile columns whose grown
// x-range meets the ellipse's x-extent inside the row's grown y-strip.  The per-Gaussian
// constants are formed once (CullGauss); every step is an explicitly rounded operation,
// so the projection (which counts the tiles) and the emission (which lists them) agree
// exactly.  Tile sides are powers of two, so their reciprocals are exact.
struct CullGauss {
    float mx, my, vx, vy;   // mean and image velocity
    float k01, det;         // conic cross term, conic determinant
    float ik00, kt;         // 1 / k00, k00 thr
    float vmax, vr;         // the ellipse's half-height, the v of its right-most point
    bool ok;                // false: the Gaussian can reach 1/255 nowhere
};

__device__ __forceinline__ CullGauss cull_setup(float mx, float my, float vx, float vy, float k00, float k01,
                                                float k11, float op) {
    CullGauss G;
    G.mx = mx;
    G.my = my;
    G.vx = vx;
    G.vy = vy;
    G.k01 = k01;
    const float thr = __fmaf_rn(__fmul_rn(2.f, logf(__fmul_rn(255.f, op))), 1.002f, 2e-3f);
    G.det = __fsub_rn(__fmul_rn(k00, k11), __fmul_rn(k01, k01));
    G.ok = thr > 0.f && G.det > 0.f && k00 > 0.f && k11 > 0.f;
    const float idet = __frcp_rn(G.det);
    G.ik00 = __frcp_rn(k00);
    G.kt = __fmul_rn(k00, thr);
    G.vmax = sqrtf(fmaxf(__fmul_rn(G.kt, idet), 0.f));
    const float uext = sqrtf(fmaxf(__fmul_rn(__fmul_rn(thr, k11), idet), 0.f));
    G.vr = __fmul_rn(__fmul_rn(-k01, uext), __frcp_rn(k11));
    return G;
}

// The kept columns [*ca, *cb) of tile row ty within the box columns [x0, x1).
__device__ __forceinline__ void cull_row_cols(const SensorDev& S, const CullGauss& G, int ty, int x0, int x1,
                                              int* ca, int* cb) {
    *ca = *cb = x0;
    if (!G.ok) return;
    const float iH = __frcp_rn((float)S.height);
    const float y0 = __fadd_rn((float)(ty * S.tile_h), 0.5f);
    const float y1 = __fadd_rn((float)min(ty * S.tile_h + S.tile_h, S.height), -0.5f);
    const float t0 = __fmaf_rn(__fmaf_rn(y0, iH, -0.5f), S.rs, S.dt);
    const float t1 = __fmaf_rn(__fmaf_rn(y1, iH, -0.5f), S.rs, S.dt);
    const float tm = __fmul_rn(0.5f, __fadd_rn(t0, t1)), ht = __fmul_rn(0.5f, fabsf(__fsub_rn(t1, t0)));
    const float cx = __fmaf_rn(G.vx, tm, G.mx), cy = __fmaf_rn(G.vy, tm, G.my);
    const float gx = __fmaf_rn(fabsf(G.vx), ht, 2e-3f), gy = __fmaf_rn(fabsf(G.vy), ht, 2e-3f);
    // the row's strip within the ellipse's v-range, relative to the moved mean
    const float va = fmaxf(__fsub_rn(__fsub_rn(y0, gy), cy), -G.vmax);
    const float vb = fminf(__fsub_rn(__fadd_rn(y1, gy), cy), G.vmax);
    if (!(va <= vb)) return;
    // x-extent over the strip: the boundary u(v) = (-k01 v +- sqrt(k00 thr - det v^2)) / k00
    // is concave (right) / convex (left) with its extreme at v = -+k01 u_ext / k11
    const float vR = fminf(fmaxf(G.vr, va), vb), vL = fminf(fmaxf(-G.vr, va), vb);
    const float rR = sqrtf(fmaxf(__fsub_rn(G.kt, __fmul_rn(G.det, __fmul_rn(vR, vR))), 0.f));
    const float rL = sqrtf(fmaxf(__fsub_rn(G.kt, __fmul_rn(G.det, __fmul_rn(vL, vL))), 0.f));
    const float uhi = __fmul_rn(__fmaf_rn(-G.k01, vR, rR), G.ik00);
    const float ulo = __fmul_rn(__fsub_rn(__fmul_rn(-G.k01, vL), rL), G.ik00);
    // tile tx is kept iff tx tw + 0.5 - gx <= cx + uhi and (its last pixel centre) + gx >= cx + ulo
    const float xh = __fadd_rn(__fadd_rn(cx, uhi), gx), xl = __fsub_rn(__fadd_rn(cx, ulo), gx);
    if (!(xl <= __fadd_rn((float)S.width, -0.5f)) || !(xh >= 0.5f)) return;
    const float itw = __frcp_rn((float)S.tile_w);
    const float fb = floorf(__fmul_rn(__fadd_rn(xh, -0.5f), itw)) + 1.f;
    const float fa = ceilf(__fmaf_rn(__fadd_rn(xl, 0.5f), itw, -1.f));
    const int a = (int)fminf(fmaxf(fa, (float)x0), (float)x1), b = (int)fminf(fmaxf(fb, (float)x0), (float)x1);
    if (a < b) {
        *ca = a;
        *cb = b;
    }
}

__device__ __forceinline__ int sensor_of_block(const Frame& fr, int block, bool lidar) {
    const int n = lidar ? fr.n_lids : fr.n_cams;
    const int* list = lidar ? fr.lid_sensors : fr.cam_sensors;
    int s = list[0];
    for (int k = 1; k < n; k++) {
        if (fr.s[list[k]].block_base <= block) s = list[k];
    }
    return s;
}

}  // namespace splat
