// project.cu -- per-Gaussian projection into every sensor of a frame, and its
// backward (chain rule to means, scales, quaternions, opacities, velocities).
//
// Camera: paper Sec. 3.2 (perspective projection, Sigma^I = J^I Sigma^C J^I^T, the
// rectangular 3-sigma AABB widened by |v^I| t_rs / 2, 16x16 tiles), Eq. (pixel velocity)
// with App. D, Eq. (alpha) for the compensated opacity.
// Lidar: Sec. 3.3 Eq. (spherical projection), J^S, v^S = J^S(-w x mu - v + v_dyn), AABB
// widened by the first two components of v^S t_rs / 2, App. A.1 azimuth tile limits with
// wrap-around and the elevation loop over sorted tile boundaries.
//
// One thread per Gaussian loops over the frame's sensors, so the Gaussian's parameters
// and its world covariance are read and formed once per frame; the outputs are
// structure-of-arrays float4 streams, so every store of a warp is one contiguous 512 B
// segment.
#include "types.cuh"

namespace splat {

struct GaussLocal {
    float3 mean, vel;
    float s[3];
    float q[4];      // normalised
    float qnorm;
    float Rq[9];
    Sym3 Sig;        // world covariance
    float opac;
};

__device__ __forceinline__ void load_gaussian(const GaussIn& g, int64_t i, GaussLocal& L) {
    L.mean = make_float3(g.means[3 * i], g.means[3 * i + 1], g.means[3 * i + 2]);
    L.s[0] = g.scales[3 * i];
    L.s[1] = g.scales[3 * i + 1];
    L.s[2] = g.scales[3 * i + 2];
    const float4 q = reinterpret_cast<const float4*>(g.quats)[i];
    L.qnorm = sqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
    const float inv = 1.0f / L.qnorm;
    L.q[0] = q.x * inv;
    L.q[1] = q.y * inv;
    L.q[2] = q.z * inv;
    L.q[3] = q.w * inv;
    quat_to_rot(L.q[0], L.q[1], L.q[2], L.q[3], L.Rq);
    // Sigma = M M^T with M = Rq diag(s)
    float M[9];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) M[3 * r + c] = L.Rq[3 * r + c] * L.s[c];
    L.Sig.xx = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
    L.Sig.xy = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
    L.Sig.xz = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
    L.Sig.yy = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
    L.Sig.yz = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
    L.Sig.zz = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
    L.opac = g.opac[i];
    L.vel = g.vel ? make_float3(g.vel[3 * i], g.vel[3 * i + 1], g.vel[3 * i + 2]) : make_float3(0.f, 0.f, 0.f);
}

__device__ __forceinline__ float3 xform(const float* R, const float* t, float3 p) {
    return make_float3(R[0] * p.x + R[1] * p.y + R[2] * p.z + t[0], R[3] * p.x + R[4] * p.y + R[5] * p.z + t[1],
                       R[6] * p.x + R[7] * p.y + R[8] * p.z + t[2]);
}
__device__ __forceinline__ float3 rot(const float* R, float3 p) {
    return make_float3(R[0] * p.x + R[1] * p.y + R[2] * p.z, R[3] * p.x + R[4] * p.y + R[5] * p.z,
                       R[6] * p.x + R[7] * p.y + R[8] * p.z);
}
__device__ __forceinline__ float3 rot_t(const float* R, float3 p) {
    return make_float3(R[0] * p.x + R[3] * p.y + R[6] * p.z, R[1] * p.x + R[4] * p.y + R[7] * p.z,
                       R[2] * p.x + R[5] * p.y + R[8] * p.z);
}
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Relative velocity of a Gaussian in the sensor frame: -w x m - v + R v_g (App. D, with
// the actor velocity term given directly as a per-Gaussian world velocity).
__device__ __forceinline__ float3 rel_velocity(const SensorDev& S, float3 m, float3 vg) {
    const float3 wxm = cross(make_float3(S.w[0], S.w[1], S.w[2]), m);
    const float3 rv = rot(S.R, vg);
    return make_float3(-wxm.x - S.v[0] + rv.x, -wxm.y - S.v[1] + rv.y, -wxm.z - S.v[2] + rv.z);
}

// 2-D covariance from the first two rows of a Jacobian (J0, J1 are 3-vectors).
__device__ __forceinline__ void cov2d(const float* J0, const float* J1, const Sym3& Sc, float& a, float& b,
                                      float& c) {
    float u0[3], u1[3];
#pragma unroll
    for (int j = 0; j < 3; j++) {
        u0[j] = J0[0] * sym_get(Sc, 0, j) + J0[1] * sym_get(Sc, 1, j) + J0[2] * sym_get(Sc, 2, j);
        u1[j] = J1[0] * sym_get(Sc, 0, j) + J1[1] * sym_get(Sc, 1, j) + J1[2] * sym_get(Sc, 2, j);
    }
    a = u0[0] * J0[0] + u0[1] * J0[1] + u0[2] * J0[2];
    b = u0[0] * J1[0] + u0[1] * J1[1] + u0[2] * J1[2];
    c = u1[0] * J1[0] + u1[1] * J1[1] + u1[2] * J1[2];
}

struct CamJ {
    float z, ux, uy, L_x, L_y;
    bool clamp_x, clamp_y;
    float J0[3], J1[3];
};

__device__ __forceinline__ void camera_jacobian(const SensorDev& S, float3 m, CamJ& cj) {
    cj.z = m.z;
    cj.ux = m.x / m.z;
    cj.uy = m.y / m.z;
    cj.L_x = fminf(fmaxf(cj.ux, -S.lim_x), S.lim_x);
    cj.L_y = fminf(fmaxf(cj.uy, -S.lim_y), S.lim_y);
    cj.clamp_x = cj.L_x != cj.ux;
    cj.clamp_y = cj.L_y != cj.uy;
    const float tx = m.z * cj.L_x, ty = m.z * cj.L_y;
    const float z2 = m.z * m.z;
    cj.J0[0] = S.fx / m.z;
    cj.J0[1] = 0.f;
    cj.J0[2] = -S.fx * tx / z2;
    cj.J1[0] = 0.f;
    cj.J1[1] = S.fy / m.z;
    cj.J1[2] = -S.fy * ty / z2;
}

struct LidJ {
    float x, y, z, rho2, rho, r2, r;
    float J[9];
};

__device__ __forceinline__ void lidar_jacobian(float3 m, LidJ& lj) {
    lj.x = m.x;
    lj.y = m.y;
    lj.z = m.z;
    lj.rho2 = m.x * m.x + m.y * m.y;
    lj.rho = sqrtf(lj.rho2);
    lj.r2 = lj.rho2 + m.z * m.z;
    lj.r = sqrtf(lj.r2);
    const float h = lj.r2 * lj.rho;
    lj.J[0] = -m.y / lj.rho2;
    lj.J[1] = m.x / lj.rho2;
    lj.J[2] = 0.f;
    lj.J[3] = -m.x * m.z / h;
    lj.J[4] = -m.y * m.z / h;
    lj.J[5] = lj.rho / lj.r2;
    lj.J[6] = m.x / lj.r;
    lj.J[7] = m.y / lj.r;
    lj.J[8] = m.z / lj.r;
}

__device__ bool project_camera(const SensorDev& S, const GaussLocal& G, float4& r0, float4& r1, float4& r2,
                               short4& rect, int& nt) {
    const float3 m = xform(S.R, S.t, G.mean);
    if (!(m.z >= S.near_plane)) return false;
    const Sym3 Sc = rotate_sym(S.R, G.Sig);
    CamJ cj;
    camera_jacobian(S, m, cj);
    float a, b, c;
    cov2d(cj.J0, cj.J1, Sc, a, b, c);
    const float A = a + S.eps, C = c + S.eps;
    const float det0 = a * c - b * b, det1 = A * C - b * b;
    if (!(det1 > 0.f)) return false;
    const float comp = sqrtf(fmaxf(det0, 0.f) / det1);
    const float op = G.opac * comp;
    if (!(op >= kAlphaMin)) return false;
    const float3 w = rel_velocity(S, m, G.vel);
    const float vx = cj.J0[0] * w.x + cj.J0[2] * w.z;
    const float vy = cj.J1[1] * w.y + cj.J1[2] * w.z;
    const float mx = S.fx * cj.ux + S.cx, my = S.fy * cj.uy + S.cy;
    const float tspan = 0.5f * S.rs + fabsf(S.dt);
    const float k = support_sigmas(S, op);
    const float ex = k * sqrtf(A) + fabsf(vx) * tspan;
    const float ey = k * sqrtf(C) + fabsf(vy) * tspan;
    const float fx0 = fminf(fmaxf(floorf((mx - ex) / S.tile_w), 0.f), (float)S.tiles_x);
    const float fx1 = fminf(fmaxf(ceilf((mx + ex) / S.tile_w), 0.f), (float)S.tiles_x);
    const float fy0 = fminf(fmaxf(floorf((my - ey) / S.tile_h), 0.f), (float)S.tiles_y);
    const float fy1 = fminf(fmaxf(ceilf((my + ey) / S.tile_h), 0.f), (float)S.tiles_y);
    const int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
    if (x1 <= x0 || y1 <= y0) return false;
    // (with the camera tile cull, support flag 4, the binning drops the box tiles where
    // alpha cannot reach 1/255; n_tiles stays the box's tile count)
    nt = (x1 - x0) * (y1 - y0);
    r0 = make_float4(mx, my, vx, vy);
    r1 = make_float4(C / det1, -b / det1, A / det1, op);
    r2 = make_float4(m.z, 0.f, 0.f, 0.f);
    rect = make_short4((short)x0, (short)y0, (short)x1, (short)y1);
    return true;
}

__device__ bool project_lidar(const SensorDev& S, const GaussLocal& G, float4& r0, float4& r1, float4& r2,
                              short4& rect, int& nt) {
    const float3 m = xform(S.R, S.t, G.mean);
    LidJ lj;
    lidar_jacobian(m, lj);
    if (!(lj.r >= S.rmin)) return false;
    if (!(lj.rho >= 1e-6f * lj.r)) return false;
    float phi = atan2f(m.y, m.x);
    if (phi < 0.f) phi += kTwoPi;
    const float om = asinf(fminf(fmaxf(m.z / lj.r, -1.f), 1.f));
    const Sym3 Sc = rotate_sym(S.R, G.Sig);
    float a, b, c;
    cov2d(lj.J, lj.J + 3, Sc, a, b, c);
    const float A = a + S.eps, C = c + S.eps;
    const float det0 = a * c - b * b, det1 = A * C - b * b;
    if (!(det1 > 0.f)) return false;
    const float comp = sqrtf(fmaxf(det0, 0.f) / det1);
    const float op = G.opac * comp;
    if (!(op >= kAlphaMin)) return false;
    const float3 w = rel_velocity(S, m, G.vel);
    const float vphi = lj.J[0] * w.x + lj.J[1] * w.y;
    const float vom = lj.J[3] * w.x + lj.J[4] * w.y + lj.J[5] * w.z;
    const float vr = lj.J[6] * w.x + lj.J[7] * w.y + lj.J[8] * w.z;
    const float half = 0.5f * S.sweep;
    const float k = support_sigmas(S, op);
    const float es = k * sqrtf(A), eos = k * sqrtf(C);
    const float ep = es + fabsf(vphi) * half;
    const float eo = eos + fabsf(vom) * half;
    float plo = phi - ep, phi_hi = phi + ep;
    float olo = om - eo, ohi = om + eo;
    if ((S.support & 2) && plo >= 0.f && phi_hi < kTwoPi) {
        // motion margins from the grid rays' own fire times t(phi) = c phi - t_sweep / 2:
        // the azimuth test |phi - phi_mean - v_phi t(phi)| <= e_phi holds for phi - phi_mean in
        // [v_phi t_m - e_phi, v_phi t_m + e_phi] / (1 - c v_phi); the elevation margin needs
        // only the times of that azimuth range.  A box across the seam keeps its margins.
        const float c = S.sweep / ((float)S.naz * S.az_res), den = 1.f - c * vphi;
        if (den > 0.f) {
            const float tm = c * phi - half;
            plo = fmaxf(plo, phi + (vphi * tm - es) / den);
            phi_hi = fminf(phi_hi, phi + (vphi * tm + es) / den);
            const float t0 = fmaxf(c * plo - half, -half), t1 = fminf(c * phi_hi - half, half);
            const float w0 = vom * t0, w1 = vom * t1;
            olo = fmaxf(olo, om - eos + fminf(w0, w1));
            ohi = fminf(ohi, om + eos + fmaxf(w0, w1));
            if (!(phi_hi >= plo) || !(ohi >= olo)) return false;
        }
    }
    // elevation rows (App. A.1): row containing omega_low .. one past the row of omega_high
    const int Mw = S.nb / S.tile_h;
    if (!(ohi > elev_bound(S, 0)) || !(olo < elev_bound(S, Mw))) return false;
    int Olo = 0, Ohi = 0;
    for (int k = 1; k < Mw; k++)
        if (elev_bound(S, k) <= olo) Olo = k;
    for (int k = 0; k < Mw; k++)
        if (elev_bound(S, k) < ohi) Ohi = k + 1;
    // azimuth columns (App. A.1), wrapped into [0, M_phi) after the span is clamped
    const int Mphi = S.tiles_x;
    const float L = plo >= 0.f ? floorf(plo / S.wphi) : floorf((plo + kTwoPi - S.phimax) / S.wphi);
    const float H = phi_hi <= kTwoPi ? ceilf(phi_hi / S.wphi) : ceilf(fmodf(phi_hi, kTwoPi) / S.wphi) + (float)Mphi;
    const float span = fminf(H - L, (float)Mphi);
    if (!(span >= 1.f) || Ohi <= Olo) return false;
    const float Lm = L - (float)Mphi * floorf(L / (float)Mphi);
    const int x0 = min(max((int)Lm, 0), Mphi - 1);
    const int x1 = x0 + (int)span;
    r0 = make_float4(phi, om, vphi, vom);
    r1 = make_float4(C / det1, -b / det1, A / det1, op);
    r2 = make_float4(lj.r, vr, 0.f, 0.f);
    rect = make_short4((short)x0, (short)Olo, (short)x1, (short)Ohi);
    nt = (x1 - x0) * (Ohi - Olo);
    return true;
}

// Every geometric parameter of Gaussian i (mean, scale, quaternion, opacity, velocity)
// is a finite number.
__device__ __forceinline__ bool finite_params(const GaussIn& g, int64_t i) {
    bool ok = isfinite(g.opac[i]);
#pragma unroll
    for (int k = 0; k < 3; k++) ok &= isfinite(g.means[3 * i + k]) && isfinite(g.scales[3 * i + k]);
    const float4 q = reinterpret_cast<const float4*>(g.quats)[i];
    ok &= isfinite(q.x) && isfinite(q.y) && isfinite(q.z) && isfinite(q.w);
    if (g.vel) {
#pragma unroll
        for (int k = 0; k < 3; k++) ok &= isfinite(g.vel[3 * i + k]);
    }
    return ok;
}

__global__ void __launch_bounds__(256) k_project(GaussIn g, const __grid_constant__ Frame fr, ProjOut out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    GaussLocal G;
    load_gaussian(g, i, G);
    // a Gaussian with a non-finite parameter (or a zero quaternion) is culled from every
    // sensor: no tile, no record, no gradient
    bool finite = finite_params(g, i) && isfinite(G.q[0]);
    for (int s = 0; s < fr.n_sensors; s++) {
        const SensorDev& S = fr.s[s];
        float4 r0, r1, r2;
        short4 rc;
        int nt = 0;
        const bool vis = finite && (S.kind == SPLAT_SENSOR_CAMERA ? project_camera(S, G, r0, r1, r2, rc, nt)
                                                                  : project_lidar(S, G, r0, r1, r2, rc, nt));
        if (vis) {
            out.rec[rec_index(s, 0, g.n, i)] = r0;
            out.rec[rec_index(s, 1, g.n, i)] = r1;
            out.rec[rec_index(s, 2, g.n, i)] = r2;
            out.rect[(size_t)s * g.n + i] = rc;
        }
        out.n_tiles[(size_t)s * g.n + i] = vis ? nt : 0;
    }
}

// ------------------------------------------------------------------------------------
// Backward.  grad layout = rec layout: g0 = d(mean_a, mean_b, v_a, v_b),
// g1 = d(conic a, b, c, o'), g2 = d(depth, v_r, -, -).
// ------------------------------------------------------------------------------------

// d(conic, o') -> gradients of the 2-D covariance parameters (a, b, c) of J Sigma J^T.
// conic = (Sigma_2d + eps I)^-1: with K the conic matrix and G its gradient written as a
// symmetric matrix, dL/d(Sigma') = -K G K.
__device__ __forceinline__ void cov2d_backward(float a, float b, float c, float eps, float opac, float4 g1,
                                               float& da, float& db, float& dc, float& dopac) {
    const float A = a + eps, C = c + eps;
    const float det1 = A * C - b * b, det0 = a * c - b * b;
    const float k00 = C / det1, k01 = -b / det1, k11 = A / det1;
    const float g00 = g1.x, g01 = 0.5f * g1.y, g11 = g1.z;
    // (K G) then (K G K)
    const float t00 = k00 * g00 + k01 * g01, t01 = k00 * g01 + k01 * g11;
    const float t10 = k01 * g00 + k11 * g01, t11 = k01 * g01 + k11 * g11;
    const float m00 = t00 * k00 + t01 * k01, m01 = t00 * k01 + t01 * k11, m11 = t10 * k01 + t11 * k11;
    da = -m00;
    dc = -m11;
    db = -2.f * m01;
    // compensation sqrt(det0 / det1) scales the opacity
    const float comp = sqrtf(fmaxf(det0, 0.f) / det1);
    dopac = g1.w * comp;
    if (det0 > 0.f && comp > 0.f) {
        const float dcomp = g1.w * opac;
        const float dq = dcomp / (2.f * comp) / (det1 * det1);
        da += dq * (c * det1 - det0 * C);
        dc += dq * (a * det1 - det0 * A);
        db += dq * (2.f * b * (det0 - det1));
    }
}

// dL/dSigma_c (full-matrix convention) and dL/dJ rows 0,1 from d(a, b, c), where
// (a, b, c) = (J0 S J0, J0 S J1, J1 S J1).
__device__ __forceinline__ void cov2d_jac_backward(const float* J0, const float* J1, const Sym3& Sc, float da,
                                                   float db, float dc, float* dSc, float* dJ0, float* dJ1) {
    const float g00 = da, g01 = 0.5f * db, g11 = dc;
#pragma unroll
    for (int p = 0; p < 3; p++)
#pragma unroll
        for (int q = 0; q < 3; q++)
            dSc[3 * p + q] = J0[p] * (g00 * J0[q] + g01 * J1[q]) + J1[p] * (g01 * J0[q] + g11 * J1[q]);
    // dJ = 2 G J Sc
    float u0[3], u1[3];
#pragma unroll
    for (int q = 0; q < 3; q++) {
        u0[q] = J0[0] * sym_get(Sc, 0, q) + J0[1] * sym_get(Sc, 1, q) + J0[2] * sym_get(Sc, 2, q);
        u1[q] = J1[0] * sym_get(Sc, 0, q) + J1[1] * sym_get(Sc, 1, q) + J1[2] * sym_get(Sc, 2, q);
    }
#pragma unroll
    for (int q = 0; q < 3; q++) {
        dJ0[q] += 2.f * (g00 * u0[q] + g01 * u1[q]);
        dJ1[q] += 2.f * (g01 * u0[q] + g11 * u1[q]);
    }
}

// Accumulate one sensor's contribution to dL/dmean (world), dL/dSigma (world, full
// matrix), dL/dopacity and dL/dvelocity.
// Sensor-parameter terms of one (sensor, Gaussian) pair, from the sensor-frame mean m, its
// total gradient dm, the covariance Sc and its gradient dSc, and dL/dw of the relative
// velocity w = -omega x m - v_s + R v_g:
//   [0..2] dL/dv_s = -dw, [3..5] dL/domega = dw x m, [6..8] dL/dt = dm (m = R mu + t),
//   [9..11] rotation R <- (I + [theta]x) R: (m - t) x dm + (R v_g) x dw + 2 axial(Sc G - G Sc),
//   G the symmetric part of dSc.
__device__ __forceinline__ void sensor_terms(const SensorDev& S, const float3 m, const Sym3& Sc, const float (&dSc)[9],
                                             const float3 dm, const float3 dw, const float3 vg, float (&ds)[12]) {
    const float3 dwxm = cross(dw, m);
    ds[0] = -dw.x;
    ds[1] = -dw.y;
    ds[2] = -dw.z;
    ds[3] = dwxm.x;
    ds[4] = dwxm.y;
    ds[5] = dwxm.z;
    ds[6] = dm.x;
    ds[7] = dm.y;
    ds[8] = dm.z;
    const float3 a = make_float3(m.x - S.t[0], m.y - S.t[1], m.z - S.t[2]);
    const float3 c1 = cross(a, dm), c2 = cross(rot(S.R, vg), dw);
    const float Sm[9] = {Sc.xx, Sc.xy, Sc.xz, Sc.xy, Sc.yy, Sc.yz, Sc.xz, Sc.yz, Sc.zz};
    float M[9];
#pragma unroll
    for (int p = 0; p < 3; p++)
#pragma unroll
        for (int q = 0; q < 3; q++) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < 3; k++) acc += Sm[3 * p + k] * 0.5f * (dSc[3 * k + q] + dSc[3 * q + k]);
            M[3 * p + q] = acc;
        }
    ds[9] = c1.x + c2.x + 2.f * (M[5] - M[7]);
    ds[10] = c1.y + c2.y + 2.f * (M[6] - M[2]);
    ds[11] = c1.z + c2.z + 2.f * (M[1] - M[3]);
}

__device__ void camera_backward(const SensorDev& S, const GaussLocal& G, float4 g0, float4 g1, float3& dmean,
                                float* dSw, float& dop, float3& dvel, bool want_sensor, float (&dsens)[12]) {
    const float3 m = xform(S.R, S.t, G.mean);
    const Sym3 Sc = rotate_sym(S.R, G.Sig);
    CamJ cj;
    camera_jacobian(S, m, cj);
    float a, b, c;
    cov2d(cj.J0, cj.J1, Sc, a, b, c);
    const float3 w = rel_velocity(S, m, G.vel);
    float da, db, dc, dopac;
    cov2d_backward(a, b, c, S.eps, G.opac, g1, da, db, dc, dopac);
    dop += dopac;
    float dSc[9], dJ0[3] = {0.f, 0.f, 0.f}, dJ1[3] = {0.f, 0.f, 0.f};
    cov2d_jac_backward(cj.J0, cj.J1, Sc, da, db, dc, dSc, dJ0, dJ1);
    // velocity v = J w (two rows)
    const float wv[3] = {w.x, w.y, w.z};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        dJ0[k] += g0.z * wv[k];
        dJ1[k] += g0.w * wv[k];
    }
    const float3 dw = make_float3(cj.J0[0] * g0.z, cj.J1[1] * g0.w, cj.J0[2] * g0.z + cj.J1[2] * g0.w);
    // mean: (fx x/z + cx, fy y/z + cy)
    const float z = m.z, iz = 1.f / z, iz2 = iz * iz;
    const float dux = S.fx * g0.x, duy = S.fy * g0.y;
    float3 dm = make_float3(dux * iz, duy * iz, -(dux * cj.ux + duy * cj.uy) * iz);
    // J entries
    dm.z += -S.fx * iz2 * dJ0[0] - S.fy * iz2 * dJ1[1];
    if (!cj.clamp_x) {
        dm.x += -S.fx * iz2 * dJ0[2];
        dm.z += 2.f * S.fx * m.x * iz2 * iz * dJ0[2];
    } else {
        dm.z += S.fx * cj.L_x * iz2 * dJ0[2];
    }
    if (!cj.clamp_y) {
        dm.y += -S.fy * iz2 * dJ1[2];
        dm.z += 2.f * S.fy * m.y * iz2 * iz * dJ1[2];
    } else {
        dm.z += S.fy * cj.L_y * iz2 * dJ1[2];
    }
    // w = -omega x m - v + R v_g
    const float3 oxdw = cross(make_float3(S.w[0], S.w[1], S.w[2]), dw);
    dm.x += oxdw.x;
    dm.y += oxdw.y;
    dm.z += oxdw.z;
    if (want_sensor) sensor_terms(S, m, Sc, dSc, dm, dw, G.vel, dsens);
    const float3 dvg = rot_t(S.R, dw);
    dvel.x += dvg.x;
    dvel.y += dvg.y;
    dvel.z += dvg.z;
    const float3 dmw = rot_t(S.R, dm);
    dmean.x += dmw.x;
    dmean.y += dmw.y;
    dmean.z += dmw.z;
    // Sigma_c = R Sigma R^T -> dSigma += R^T dSc R
    float T[9];
#pragma unroll
    for (int p = 0; p < 3; p++)
#pragma unroll
        for (int q = 0; q < 3; q++) T[3 * p + q] = S.R[p] * dSc[q] + S.R[3 + p] * dSc[3 + q] + S.R[6 + p] * dSc[6 + q];
#pragma unroll
    for (int p = 0; p < 3; p++)
#pragma unroll
        for (int q = 0; q < 3; q++) dSw[3 * p + q] += T[3 * p] * S.R[q] + T[3 * p + 1] * S.R[3 + q] + T[3 * p + 2] * S.R[6 + q];
}

__device__ void lidar_backward(const SensorDev& S, const GaussLocal& G, float4 g0, float4 g1, float4 g2,
                               float3& dmean, float* dSw, float& dop, float3& dvel, bool want_sensor,
                               float (&dsens)[12]) {
    const float3 m = xform(S.R, S.t, G.mean);
    const Sym3 Sc = rotate_sym(S.R, G.Sig);
    LidJ lj;
    lidar_jacobian(m, lj);
    const float* J = lj.J;
    float a, b, c;
    cov2d(J, J + 3, Sc, a, b, c);
    const float3 w = rel_velocity(S, m, G.vel);
    float da, db, dc, dopac;
    cov2d_backward(a, b, c, S.eps, G.opac, g1, da, db, dc, dopac);
    dop += dopac;
    float dSc[9], dJ[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    cov2d_jac_backward(J, J + 3, Sc, da, db, dc, dSc, dJ, dJ + 3);
    // v^S = J w (three rows)
    const float dv[3] = {g0.z, g0.w, g2.y};
    const float wv[3] = {w.x, w.y, w.z};
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int k = 0; k < 3; k++) dJ[3 * r + k] += dv[r] * wv[k];
    const float3 dw = make_float3(J[0] * dv[0] + J[3] * dv[1] + J[6] * dv[2], J[1] * dv[0] + J[4] * dv[1] + J[7] * dv[2],
                                  J[2] * dv[0] + J[5] * dv[1] + J[8] * dv[2]);
    // mean (phi, omega, r): the rows of J are their gradients
    const float ds[3] = {g0.x, g0.y, g2.x};
    float3 dm = make_float3(J[0] * ds[0] + J[3] * ds[1] + J[6] * ds[2], J[1] * ds[0] + J[4] * ds[1] + J[7] * ds[2],
                            J[2] * ds[0] + J[5] * ds[1] + J[8] * ds[2]);
    // second derivatives: d J_e / d m
    const float x = lj.x, y = lj.y, z = lj.z, rho = lj.rho, rho2 = lj.rho2, r2 = lj.r2, r = lj.r;
    const float rho4 = rho2 * rho2;
    dm.x += dJ[0] * (2.f * x * y / rho4) + dJ[1] * ((y * y - x * x) / rho4);
    dm.y += dJ[0] * ((y * y - x * x) / rho4) + dJ[1] * (-2.f * x * y / rho4);
    const float h = r2 * rho, h2 = h * h;
    const float dhx = 2.f * x * rho + r2 * x / rho, dhy = 2.f * y * rho + r2 * y / rho, dhz = 2.f * z * rho;
    dm.x += dJ[3] * (-z / h + x * z * dhx / h2) + dJ[4] * (y * z * dhx / h2);
    dm.y += dJ[3] * (x * z * dhy / h2) + dJ[4] * (-z / h + y * z * dhy / h2);
    dm.z += dJ[3] * (-x / h + x * z * dhz / h2) + dJ[4] * (-y / h + y * z * dhz / h2);
    const float r4 = r2 * r2;
    dm.x += dJ[5] * ((x / rho) / r2 - 2.f * x * rho / r4);
    dm.y += dJ[5] * ((y / rho) / r2 - 2.f * y * rho / r4);
    dm.z += dJ[5] * (-2.f * z * rho / r4);
    const float r3 = r2 * r;
    const float mv[3] = {x, y, z};
    float dmm[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int e = 0; e < 3; e++)
#pragma unroll
        for (int k = 0; k < 3; k++) dmm[k] += dJ[6 + e] * ((e == k ? 1.f / r : 0.f) - mv[e] * mv[k] / r3);
    dm.x += dmm[0];
    dm.y += dmm[1];
    dm.z += dmm[2];
    const float3 oxdw = cross(make_float3(S.w[0], S.w[1], S.w[2]), dw);
    dm.x += oxdw.x;
    dm.y += oxdw.y;
    dm.z += oxdw.z;
    if (want_sensor) sensor_terms(S, m, Sc, dSc, dm, dw, G.vel, dsens);
    const float3 dvg = rot_t(S.R, dw);
    dvel.x += dvg.x;
    dvel.y += dvg.y;
    dvel.z += dvg.z;
    const float3 dmw = rot_t(S.R, dm);
    dmean.x += dmw.x;
    dmean.y += dmw.y;
    dmean.z += dmw.z;
    float T[9];
#pragma unroll
    for (int p = 0; p < 3; p++)
#pragma unroll
        for (int q = 0; q < 3; q++) T[3 * p + q] = S.R[p] * dSc[q] + S.R[3 + p] * dSc[3 + q] + S.R[6 + p] * dSc[6 + q];
#pragma unroll
    for (int p = 0; p < 3; p++)
#pragma unroll
        for (int q = 0; q < 3; q++) dSw[3 * p + q] += T[3 * p] * S.R[q] + T[3 * p + 1] * S.R[3 + q] + T[3 * p + 2] * S.R[6 + q];
}

__global__ void __launch_bounds__(256) k_project_backward(GaussIn g, const __grid_constant__ Frame fr,
                                                          const int32_t* __restrict__ n_tiles,
                                                          const float4* __restrict__ grad, GradOut out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // no early exit: the optional per-sensor sums below reduce over whole warps
    bool active = i < g.n;
    bool any = false;
    if (active)
        for (int s = 0; s < fr.n_sensors; s++) any |= n_tiles[(size_t)s * g.n + i] > 0;
    active = active && any;
    if (!active && !out.sensor) return;
    GaussLocal G;
    if (active) load_gaussian(g, i, G);
    float3 dmean = make_float3(0.f, 0.f, 0.f), dvel = make_float3(0.f, 0.f, 0.f);
    float dSw[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float dop = 0.f;
    for (int s = 0; s < fr.n_sensors; s++) {
        float dsens[12];
#pragma unroll
        for (int k = 0; k < 12; k++) dsens[k] = 0.f;
        if (active && n_tiles[(size_t)s * g.n + i] > 0) {
            const SensorDev& S = fr.s[s];
            const float4 g0 = grad[rec_index(s, 0, g.n, i)];
            const float4 g1 = grad[rec_index(s, 1, g.n, i)];
            if (S.kind == SPLAT_SENSOR_CAMERA) {
                camera_backward(S, G, g0, g1, dmean, dSw, dop, dvel, out.sensor != nullptr, dsens);
            } else {
                const float4 g2 = grad[rec_index(s, 2, g.n, i)];
                lidar_backward(S, G, g0, g1, g2, dmean, dSw, dop, dvel, out.sensor != nullptr, dsens);
            }
        }
        if (out.sensor) {   // the warp's sum, one atomic per component (uniform branch)
#pragma unroll
            for (int k = 0; k < 12; k++) {
                float v = dsens[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                // slots: velocities 0..5, (6: camera time offset), translation 8..10, rotation 11..13
                if ((threadIdx.x & 31) == 0 && v != 0.f) atomicAdd(out.sensor + 16 * s + (k < 6 ? k : k + 2), v);
            }
        }
    }
    if (!active) return;
    // Sigma = M M^T, M = Rq diag(s): dM = (dS + dS^T) M
    float M[9], dM[9];
#pragma unroll
    for (int p = 0; p < 3; p++)
#pragma unroll
        for (int q = 0; q < 3; q++) M[3 * p + q] = G.Rq[3 * p + q] * G.s[q];
#pragma unroll
    for (int p = 0; p < 3; p++)
#pragma unroll
        for (int q = 0; q < 3; q++) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < 3; k++) acc += (dSw[3 * p + k] + dSw[3 * k + p]) * M[3 * k + q];
            dM[3 * p + q] = acc;
        }
    float ds[3] = {0.f, 0.f, 0.f}, dR[9];
#pragma unroll
    for (int p = 0; p < 3; p++)
#pragma unroll
        for (int q = 0; q < 3; q++) {
            ds[q] += dM[3 * p + q] * G.Rq[3 * p + q];
            dR[3 * p + q] = dM[3 * p + q] * G.s[q];
        }
    // rotation entries -> normalised quaternion (w, x, y, z)
    const float qw = G.q[0], qx = G.q[1], qy = G.q[2], qz = G.q[3];
    float dq[4];
    dq[0] = 2.f * (-qz * dR[1] + qy * dR[2] + qz * dR[3] - qx * dR[5] - qy * dR[6] + qx * dR[7]);
    dq[1] = 2.f * (qy * dR[1] + qz * dR[2] + qy * dR[3] - 2.f * qx * dR[4] - qw * dR[5] + qz * dR[6] + qw * dR[7] -
                   2.f * qx * dR[8]);
    dq[2] = 2.f * (-2.f * qy * dR[0] + qx * dR[1] + qw * dR[2] + qx * dR[3] + qz * dR[5] - qw * dR[6] + qz * dR[7] -
                   2.f * qy * dR[8]);
    dq[3] = 2.f * (-2.f * qz * dR[0] - qw * dR[1] + qx * dR[2] + qw * dR[3] - 2.f * qz * dR[4] + qy * dR[5] +
                   qx * dR[6] + qy * dR[7]);
    const float dot = qw * dq[0] + qx * dq[1] + qy * dq[2] + qz * dq[3];
    const float inv = 1.f / G.qnorm;
    out.means[3 * i] += dmean.x;
    out.means[3 * i + 1] += dmean.y;
    out.means[3 * i + 2] += dmean.z;
    out.scales[3 * i] += ds[0];
    out.scales[3 * i + 1] += ds[1];
    out.scales[3 * i + 2] += ds[2];
#pragma unroll
    for (int k = 0; k < 4; k++) out.quats[4 * i + k] += (dq[k] - G.q[k] * dot) * inv;
    out.opac[i] += dop;
    if (out.vel) {
        out.vel[3 * i] += dvel.x;
        out.vel[3 * i + 1] += dvel.y;
        out.vel[3 * i + 2] += dvel.z;
    }
}

// Adds to *count the number of Gaussians with a non-finite geometric parameter (one warp
// vote and at most one atomic per warp).
__global__ void __launch_bounds__(256) k_count_nonfinite(GaussIn g, unsigned long long* count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool bad = i < g.n && !finite_params(g, i);
    const unsigned vote = __ballot_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && vote) atomicAdd(count, (unsigned long long)__popc(vote));
}

void launch_count_nonfinite(const GaussIn& g, unsigned long long* count, cudaStream_t st) {
    if (g.n == 0) return;
    const unsigned blocks = (unsigned)((g.n + 255) / 256);
    k_count_nonfinite<<<blocks, 256, 0, st>>>(g, count);
}

void launch_project(const GaussIn& g, const Frame& fr, const ProjOut& out, cudaStream_t st) {
    if (g.n == 0) return;
    const unsigned blocks = (unsigned)((g.n + 255) / 256);
    k_project<<<blocks, 256, 0, st>>>(g, fr, out);
}

void launch_project_backward(const GaussIn& g, const Frame& fr, const int32_t* n_tiles, const float4* grad,
                             const GradOut& out, cudaStream_t st) {
    if (g.n == 0) return;
    const unsigned blocks = (unsigned)((g.n + 255) / 256);
    k_project_backward<<<blocks, 256, 0, st>>>(g, fr, n_tiles, grad, out);
}

}  // namespace splat
