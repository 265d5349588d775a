/*
 * splat_oracle.c -- plain, slow FP64 reference renderer for SplatAD's camera and
 * lidar rasterizer (arXiv 2411.16816).  TEST INFRASTRUCTURE ONLY: it is used by the
 * tests, by the smoke check and by the timed CPU baseline of the benchmark, never by
 * the library's product path.  It shares no code, header or table with the CUDA
 * library; the two only consume the same seeded FP32 input arrays.
 *
 * Every ray is rendered on its own with no tiling of the work: all Gaussians whose
 * tile rectangle contains the ray's tile are collected, sorted by (depth, id) and
 * alpha-blended front to back.  Gradients are hand-written reverse mode in FP64.
 *
 * Paper passages followed (section / equation):
 *   Sec. 3.2 "Projection, tiling, and sorting"  -- camera projection, J^I, 3-sigma AABB,
 *                                                 tiles and depth order
 *   Eq. (pixel velocity) and App. D               -- v^I = J^I(-w x mu - v + v_dyn)
 *   Sec. 3.2 rolling-shutter AABB                 -- extent + |v| * t_rs / 2
 *   Eq. (t_pix), (alpha blend), (alpha), (delta)  -- camera rasterization
 *   Eq. (spherical projection) and J^S            -- lidar projection, Sec. 3.3
 *   Sec. 3.3 v^S and AABB                          -- lidar velocity and extent
 *   App. A.1 (Phi_low / Phi_high, wrap)           -- lidar azimuth tiles; elevation loop
 *   Sec. 3.3 rasterization, r_rs = r + v_r t_l    -- expected and median range
 * Readings where the paper is silent are listed in the design notes and repeated at
 * the point of use below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define TWO_PI 6.283185307179586476925286766559
#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.999
#define T_EPS 1e-4

/* ---------------------------------------------------------------------------------
 * Sensor parameter vector (double[40]); values are the FP32 inputs promoted.
 * ------------------------------------------------------------------------------- */
enum {
    P_KIND = 0,          /* 0 camera, 1 lidar */
    P_R = 1,             /* 9: world->sensor rotation, row-major */
    P_T = 10,            /* 3: translation */
    P_V = 13,            /* 3: sensor linear velocity (sensor frame) */
    P_W = 16,            /* 3: sensor angular velocity (sensor frame) */
    /* camera */
    P_WIDTH = 19, P_HEIGHT = 20, P_FX = 21, P_FY = 22, P_CX = 23, P_CY = 24,
    P_RS = 25, P_DT = 26, P_EPS = 27, P_NEAR = 28, P_TW = 29, P_TH = 30,
    /* lidar */
    P_NB = 19, P_NAZ = 20, P_AZRES = 21, P_SWEEP = 22, P_LEPS = 23, P_RMIN = 24,
    P_TAZ = 25, P_TEL = 26,
    /* both kinds */
    P_SUPPORT = 31,      /* tile extent flags: 1 = where alpha can reach 1/255 instead of 3 sigma
                          * (Sec. 3.2); 2 = lidar motion margins from the grid rays' own times;
                          * 4 = camera tile cull (a box tile where alpha cannot reach 1/255 is
                          * not listed) */
    P_ALLG = 32          /* render from every visible Gaussian, without the tile predicate */
};

/* Projected record (double[16]) */
enum {
    R_MA = 0, R_MB = 1,          /* 2-D mean: pixel (u,v) or (phi, omega) */
    R_CA = 2, R_CB = 3, R_CC = 4, /* conic of (Sigma' ) */
    R_OP = 5,                     /* compensated opacity o' */
    R_DEPTH = 6,                  /* z (camera) or range r (lidar) */
    R_VA = 7, R_VB = 8, R_VR = 9, /* sensor-space velocity */
    R_SAA = 10, R_SAB = 11, R_SBB = 12, /* Sigma' = Sigma_2d + eps I */
    R_COMP = 13, R_EXA = 14, R_EXB = 15,
    /* lidar tile box below / above the mean along azimuth (a) and elevation (b); equal to
     * the symmetric extents unless the sweep-time bounds tighten them */
    R_LA = 16, R_HA = 17, R_LB = 18, R_HB = 19
};
#define REC 20

typedef struct {
    double mean[3], S[9];       /* world mean and covariance */
    double q[4], qn, Rq[9], s[3];
    double m[3];                /* sensor-frame mean */
    double Sc[9];               /* sensor-frame covariance */
    double J[9];                /* camera: rows 0,1 used; lidar: full J^S */
    double w[3];                /* relative velocity in sensor frame */
    int clamp_x, clamp_y;       /* camera Jacobian clamp flags */
    double lim_x, lim_y;
} proj_state;

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* Distance to the nearest integer (guard bands for FP32-vs-FP64 decisions). */
static double frac_dist(double x) { return fabs(x - floor(x + 0.5)); }

/* Rotation of a normalised w-x-y-z quaternion. */
static void quat_to_rot(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* C = A B for 3x3 */
static void mm3(const double *A, const double *B, double *C) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}
/* C = A B^T */
static void mmt3(const double *A, const double *B, double *C) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * j + k];
            C[3 * i + j] = s;
        }
}
/* C = A^T B */
static void mtm3(const double *A, const double *B, double *C) {
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += A[3 * k + i] * B[3 * k + j];
            C[3 * i + j] = s;
        }
}
static void cross3(const double *a, const double *b, double *c) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* 3DGS covariance Sigma = R(q) diag(s^2) R(q)^T, then sensor frame and relative
 * velocity (Sec. 3.1, Sec. 3.2, App. D with v_dyn = R v_gauss). */
static void common_state(const double *P, const double *mean, const double *scale, const double *quat,
                         const double *vel, proj_state *st) {
    for (int k = 0; k < 3; k++) { st->mean[k] = mean[k]; st->s[k] = scale[k]; }
    double qq = 0;
    for (int k = 0; k < 4; k++) { st->q[k] = quat[k]; qq += st->q[k] * st->q[k]; }
    st->qn = sqrt(qq);
    double qh[4];
    for (int k = 0; k < 4; k++) qh[k] = st->q[k] / st->qn;
    quat_to_rot(qh, st->Rq);
    double M[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) M[3 * i + j] = st->Rq[3 * i + j] * st->s[j];
    mmt3(M, M, st->S);
    const double *R = P + P_R;
    for (int i = 0; i < 3; i++) {
        double s = P[P_T + i];
        for (int k = 0; k < 3; k++) s += R[3 * i + k] * st->mean[k];
        st->m[i] = s;
    }
    double tmp[9];
    mm3(R, st->S, tmp);
    mmt3(tmp, R, st->Sc);
    double wxm[3], vg[3] = {0, 0, 0};
    cross3(P + P_W, st->m, wxm);
    if (vel)
        for (int i = 0; i < 3; i++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += R[3 * i + k] * vel[k];
            vg[i] = s;
        }
    for (int i = 0; i < 3; i++) st->w[i] = -wxm[i] - P[P_V + i] + vg[i];
}

/* Sigma' = J2 Sc J2^T + eps I (rows 0,1 of J), conic, compensation (Eq. alpha). */
static int cov2d(const proj_state *st, double eps, double out[6]) {
    const double *J = st->J;
    double a = 0, b = 0, c = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            a += J[i] * st->Sc[3 * i + j] * J[j];
            b += J[i] * st->Sc[3 * i + j] * J[3 + j];
            c += J[3 + i] * st->Sc[3 * i + j] * J[3 + j];
        }
    double A = a + eps, C = c + eps;
    double det0 = a * c - b * b, det1 = A * C - b * b;
    if (!(det1 > 0)) return 0;
    out[0] = A; out[1] = b; out[2] = C;
    out[3] = sqrt((det0 > 0 ? det0 : 0) / det1);
    out[4] = det1;
    out[5] = det0;
    return 1;
}


/* Half-extent of the tile box in standard deviations of Sigma'.  The paper's box is
 * 3 sigma (Sec. 3.2, Sec. 3.3).  The opacity-aware alternative takes exactly the ellipse
 * where alpha = o' exp(-d^T Sigma'^-1 d / 2) can reach 1/255: d^T Sigma'^-1 d <= 2 ln(255 o'),
 * whose bounding box has half-widths sqrt(2 ln(255 o')) times the standard deviations. */
static double support_sigmas(const double *P, double op) {
    if (!((int)P[P_SUPPORT] & 1)) return 3.0;
    return op > ALPHA_MIN ? sqrt(2.0 * log(255.0 * op)) : 0.0;
}

/* Lidar motion margins from the rays' own times (an option of the tile extent).  A grid
 * ray at azimuth phi is fired at t(phi) = c phi - t_sweep / 2, c = t_sweep / (n_az az_res),
 * so the mean it sees has moved by v_phi t(phi), not by up to |v_phi| t_sweep / 2: with
 * u = phi - phi_mean, the azimuth test |u - v_phi t(phi)| <= e_phi holds for
 * u in [(v_phi t_m - e_phi), (v_phi t_m + e_phi)] / (1 - c v_phi), t_m = t(phi_mean); the
 * elevation margin then needs only the times of that azimuth range.  Both intervals are
 * intersected with the symmetric box; Gaussians whose symmetric box crosses the sweep's
 * seam at azimuth 0 (where t jumps by a whole sweep) keep it. */
static void sweep_time_box(const double *P, double e_phi, double e_om, double half, double *rec) {
    double phi = rec[R_MA], om = rec[R_MB], vphi = rec[R_VA], vom = rec[R_VB];
    double plo = phi - rec[R_EXA], phi_hi = phi + rec[R_EXA];
    double c = P[P_SWEEP] / (P[P_NAZ] * P[P_AZRES]), den = 1.0 - c * vphi;
    if (!(plo >= 0 && phi_hi < TWO_PI && den > 0)) return;
    double tm = c * phi - half;
    double lo = fmax(plo, phi + (vphi * tm - e_phi) / den);
    double hi = fmin(phi_hi, phi + (vphi * tm + e_phi) / den);
    double t0 = fmax(c * lo - half, -half), t1 = fmin(c * hi - half, half);
    double w0 = vom * t0, w1 = vom * t1;
    double olo = fmax(om - rec[R_EXB], om - e_om + fmin(w0, w1));
    double ohi = fmin(om + rec[R_EXB], om + e_om + fmax(w0, w1));
    rec[R_LA] = phi - lo;
    rec[R_HA] = hi - phi;
    rec[R_LB] = om - olo;
    rec[R_HB] = ohi - om;
}

/* Camera tile rectangle [x0,x1) x [y0,y1) from the AABB (Sec. 3.2), widened by `extra`
 * pixels on every side.  Returns 1 if an edge lies within `guard` pixels of a tile edge. */
static int camera_rect(const double *P, const double *rec, double extra, int rect[4], double guard) {
    double W = P[P_WIDTH], H = P[P_HEIGHT];
    int tw = (int)P[P_TW], th = (int)P[P_TH];
    int ntx = ((int)W + tw - 1) / tw, nty = ((int)H + th - 1) / th;
    double ea = rec[R_EXA] + extra, eb = rec[R_EXB] + extra;
    if (ea < 0 || eb < 0) { rect[0] = rect[1] = rect[2] = rect[3] = 0; return 0; }
    double xl = (rec[R_MA] - ea) / tw, xh = (rec[R_MA] + ea) / tw;
    double yl = (rec[R_MB] - eb) / th, yh = (rec[R_MB] + eb) / th;
    double gx = guard / tw, gy = guard / th;
    int m = 0;
    if (guard > 0 &&
        ((xl > -1 && xl < ntx + 1 && frac_dist(xl) < gx) || (xh > -1 && xh < ntx + 1 && frac_dist(xh) < gx) ||
         (yl > -1 && yl < nty + 1 && frac_dist(yl) < gy) || (yh > -1 && yh < nty + 1 && frac_dist(yh) < gy)))
        m = 1;
    rect[0] = (int)clampd(floor(xl), 0, ntx); rect[2] = (int)clampd(ceil(xh), 0, ntx);
    rect[1] = (int)clampd(floor(yl), 0, nty); rect[3] = (int)clampd(ceil(yh), 0, nty);
    return m;
}

/* Camera tile cull (tile-extent option 4): the margin by which a projected Gaussian misses
 * alpha >= 1/255 everywhere in tile (tx, ty).  Every pixel of the tile, at its row time
 * t (Eq. t_pix), sees the mean moved to mean + v t (Eq. delta), i.e. the pixel acts as a
 * point displaced by at most |v| (t1 - t0) / 2 per axis from the mean at the tile's
 * mid-time; so alpha = o' exp(-m / 2) (Eq. alpha, m = d^T Sigma'^-1 d) can reach 1/255 in
 * the tile only if the minimum of m over the rectangle of the tile's pixel centres grown
 * by that sweep is at most 2 ln(255 o').  The margin is that minimum, over the rectangle
 * grown by CULL_GROW more pixels, minus 2 ln(255 o') (1 + CULL_REL) - CULL_ABS: positive
 * means the pair is not listed.  The small growth and threshold margins keep every pair
 * that an FP32 evaluation of alpha could blend, so the cull never changes a render. */
#define CULL_GROW 2e-3
#define CULL_REL 2e-3
#define CULL_ABS 2e-3
static double camera_tile_margin(const double *P, const double *rec, int tx, int ty) {
    double W = P[P_WIDTH], H = P[P_HEIGHT];
    int tw = (int)P[P_TW], th = (int)P[P_TH];
    double x0 = tx * tw + 0.5, x1 = fmin((double)(tx * tw + tw), W) - 0.5;
    double y0 = ty * th + 0.5, y1 = fmin((double)(ty * th + th), H) - 0.5;
    double t0 = (y0 / H - 0.5) * P[P_RS] + P[P_DT], t1 = (y1 / H - 0.5) * P[P_RS] + P[P_DT];
    double tm = 0.5 * (t0 + t1), ht = 0.5 * fabs(t1 - t0);
    double cx = rec[R_MA] + rec[R_VA] * tm, cy = rec[R_MB] + rec[R_VB] * tm;
    double gx = fabs(rec[R_VA]) * ht + CULL_GROW, gy = fabs(rec[R_VB]) * ht + CULL_GROW;
    /* the rectangle relative to the moved mean */
    double ua = x0 - gx - cx, ub = x1 + gx - cx, va = y0 - gy - cy, vb = y1 + gy - cy;
    double a = rec[R_CA], b = rec[R_CB], c = rec[R_CC];
#define M_FORM(u, v) (a * (u) * (u) + 2 * b * (u) * (v) + c * (v) * (v))
    double mmin;
    if (ua <= 0 && ub >= 0 && va <= 0 && vb >= 0) {
        mmin = 0;   /* the mean lies in the rectangle */
    } else {
        /* a convex quadratic's minimum over a rectangle without its vertex lies on an edge;
         * on each edge it is the 1-D vertex clamped to the edge */
        double e1 = M_FORM(ua, clampd(-b * ua / c, va, vb));
        double e2 = M_FORM(ub, clampd(-b * ub / c, va, vb));
        double e3 = M_FORM(clampd(-b * va / a, ua, ub), va);
        double e4 = M_FORM(clampd(-b * vb / a, ua, ub), vb);
        mmin = fmin(fmin(e1, e2), fmin(e3, e4));
    }
#undef M_FORM
    double op = rec[R_OP];
    if (!(op > 0)) return 1e300;
    double thr = 2.0 * log(255.0 * op) * (1.0 + CULL_REL) + CULL_ABS;
    return mmin - thr;
}

static int camera_cull(const double *P) { return (int)P[P_KIND] == 0 && ((int)P[P_SUPPORT] & 4); }

/* ---------------------------------------------------------------------------------
 * Camera projection (Sec. 3.2).  Returns 1 if visible.  *marg is set when an FP32
 * evaluation could take a different discrete decision (guard band).
 * ------------------------------------------------------------------------------- */
static int project_camera(const double *P, const double *mean, const double *scale, const double *quat,
                          double opac, const double *vel, proj_state *st, double *rec, int rect[4],
                          int orect[4], int irect[4], double guard_px, int *marg) {
    common_state(P, mean, scale, quat, vel, st);
    memset(rec, 0, sizeof(double) * REC);
    for (int k = 0; k < 4; k++) rect[k] = orect[k] = irect[k] = 0;
    *marg = 0;
    int cull_marg = 0;
    double x = st->m[0], y = st->m[1], z = st->m[2];
    double nearp = P[P_NEAR];
    if (fabs(z - nearp) <= 1e-6 * fmax(fabs(nearp), 1e-3)) *marg = 1;
    if (!(z >= nearp)) return 0;
    double W = P[P_WIDTH], H = P[P_HEIGHT], fx = P[P_FX], fy = P[P_FY];
    /* Reading: Jacobian uses x/z, y/z clamped to 1.3 x tan(half field of view). */
    st->lim_x = 1.3 * 0.5 * W / fx;
    st->lim_y = 1.3 * 0.5 * H / fy;
    double ux = x / z, uy = y / z;
    double cx = clampd(ux, -st->lim_x, st->lim_x), cy = clampd(uy, -st->lim_y, st->lim_y);
    st->clamp_x = (cx != ux);
    st->clamp_y = (cy != uy);
    double tx = z * cx, ty = z * cy;
    memset(st->J, 0, sizeof(st->J));
    st->J[0] = fx / z; st->J[2] = -fx * tx / (z * z);
    st->J[4] = fy / z; st->J[5] = -fy * ty / (z * z);
    double cv[6];
    if (!cov2d(st, P[P_EPS], cv)) return 0;
    double A = cv[0], B = cv[1], C = cv[2], comp = cv[3], det1 = cv[4];
    double op = opac * comp;
    if (fabs(op - ALPHA_MIN) <= 5e-5 * ALPHA_MIN) cull_marg = 1;
    rec[R_MA] = fx * ux + P[P_CX];
    rec[R_MB] = fy * uy + P[P_CY];
    rec[R_CA] = C / det1; rec[R_CB] = -B / det1; rec[R_CC] = A / det1;
    rec[R_OP] = op;
    rec[R_DEPTH] = z;
    /* Eq. (pixel velocity): v^I = J^I w */
    rec[R_VA] = st->J[0] * st->w[0] + st->J[1] * st->w[1] + st->J[2] * st->w[2];
    rec[R_VB] = st->J[3] * st->w[0] + st->J[4] * st->w[1] + st->J[5] * st->w[2];
    rec[R_VR] = 0;
    rec[R_SAA] = A; rec[R_SAB] = B; rec[R_SBB] = C;
    rec[R_COMP] = comp;
    /* Rectangular k-sigma AABB of Sigma' plus per-component |v| (t_rs/2 + |time offset|). */
    double tspan = 0.5 * P[P_RS] + fabs(P[P_DT]);
    double k = support_sigmas(P, op);
    rec[R_EXA] = k * sqrt(A) + fabs(rec[R_VA]) * tspan;
    rec[R_EXB] = k * sqrt(C) + fabs(rec[R_VB]) * tspan;
    if (camera_rect(P, rec, 0.0, rect, guard_px)) *marg = 1;
    if (cull_marg) *marg = 1;
    if (*marg) {
        camera_rect(P, rec, guard_px, orect, 0.0);
        /* tiles inside the shrunk box belong to the Gaussian whatever the rounding */
        if (!cull_marg) camera_rect(P, rec, -guard_px, irect, 0.0);
    }
    if (op < ALPHA_MIN) return 0;
    return rect[2] > rect[0] && rect[3] > rect[1];
}

/* Elevation tile boundaries: between channels k*N-1 and k*N, outer ones half a spacing
 * beyond the first and last beams (App. A.1; reading of "between the channels"). */
static void elevation_bounds(const double *elev, int nb, int tel, double *bnd) {
    int mw = nb / tel;
    bnd[0] = elev[0] - 0.5 * ((double)elev[1] - (double)elev[0]);
    for (int k = 1; k < mw; k++) bnd[k] = 0.5 * ((double)elev[k * tel - 1] + (double)elev[k * tel]);
    bnd[mw] = elev[nb - 1] + 0.5 * ((double)elev[nb - 1] - (double)elev[nb - 2]);
}

/* Lidar azimuth tile range from App. A.1 (radians).  phi_max = M_phi N_phi res. */
static void azimuth_tiles(double plo, double phi_, double wphi, int mphi, double phimax, int *lo, int *hi) {
    double L, Hh;
    if (plo >= 0) L = floor(plo / wphi);
    else L = floor((plo + TWO_PI - phimax) / wphi);
    if (phi_ <= TWO_PI) Hh = ceil(phi_ / wphi);
    else Hh = ceil(fmod(phi_, TWO_PI) / wphi) + mphi;
    /* Reading: a span wider than the full circle covers every column once. */
    if (Hh - L > mphi) Hh = L + mphi;
    *lo = (int)L; *hi = (int)Hh;
}

/* Lidar tile rectangle: azimuth columns [Plo, Phi) (may run past either end and wrap)
 * and elevation rows [Olo, Ohi), from the AABB widened by `extra` radians.  Returns the
 * number of tiles (0 if empty); *marg is set if an edge lies within `guard` of a
 * decision boundary. */
static int lidar_rect(const double *P, const double *elev, const double *rec, double extra, int rect[4],
                      double guard, int *marg) {
    int nb = (int)P[P_NB], naz = (int)P[P_NAZ], taz = (int)P[P_TAZ], tel = (int)P[P_TEL];
    int mphi = (naz + taz - 1) / taz, mw = nb / tel;
    double wphi = taz * P[P_AZRES], phimax = mphi * wphi;
    double la = rec[R_LA] + extra, ha = rec[R_HA] + extra, lb = rec[R_LB] + extra, hb = rec[R_HB] + extra;
    rect[0] = rect[1] = rect[2] = rect[3] = 0;
    if (la + ha < 0 || lb + hb < 0) return 0;
    double plo = rec[R_MA] - la, phi_hi = rec[R_MA] + ha;
    double olo = rec[R_MB] - lb, ohi = rec[R_MB] + hb;
    double bnd[1025];
    elevation_bounds(elev, nb, tel, bnd);
    rect[0] = rect[1] = rect[2] = rect[3] = 0;
    if (guard > 0) {
        double g = guard;
        if (fabs(plo) < g || fabs(phi_hi - TWO_PI) < g) *marg = 1;
        double a1 = plo >= 0 ? plo / wphi : (plo + TWO_PI - phimax) / wphi;
        double a2 = phi_hi <= TWO_PI ? phi_hi / wphi : fmod(phi_hi, TWO_PI) / wphi;
        if (frac_dist(a1) < g / wphi || frac_dist(a2) < g / wphi) *marg = 1;
        for (int k = 0; k <= mw; k++)
            if (fabs(olo - bnd[k]) < g || fabs(ohi - bnd[k]) < g) *marg = 1;
    }
    /* Elevation loop over the sorted boundaries (App. A.1).  Reading of the garbled
     * upper rule: the lower row is the one containing omega_low, the upper (exclusive)
     * row is one past the row containing omega_high; outside the beam fan -> culled. */
    if (!(ohi > bnd[0]) || !(olo < bnd[mw])) return 0;
    int Olo = 0, Ohi = 0;
    for (int k = 1; k < mw; k++)
        if (bnd[k] <= olo) Olo = k;
    for (int k = 0; k < mw; k++)
        if (bnd[k] < ohi) Ohi = k + 1;
    int Plo, Phi;
    azimuth_tiles(plo, phi_hi, wphi, mphi, phimax, &Plo, &Phi);
    if (!(Phi > Plo && Ohi > Olo)) return 0;
    rect[0] = Plo; rect[1] = Olo; rect[2] = Phi; rect[3] = Ohi;
    return (Phi - Plo) * (Ohi - Olo);
}

/* ---------------------------------------------------------------------------------
 * Lidar projection (Sec. 3.3, App. A.1).
 * ------------------------------------------------------------------------------- */
static int project_lidar(const double *P, const double *elev, const double *mean, const double *scale,
                         const double *quat, double opac, const double *vel, proj_state *st, double *rec,
                         int rect[4], int orect[4], int irect[4], double guard_rad, int *marg) {
    common_state(P, mean, scale, quat, vel, st);
    memset(rec, 0, sizeof(double) * REC);
    for (int k = 0; k < 4; k++) rect[k] = orect[k] = irect[k] = 0;
    *marg = 0;
    int cull_marg = 0;
    double x = st->m[0], y = st->m[1], z = st->m[2];
    double rho2 = x * x + y * y, rho = sqrt(rho2), r2 = rho2 + z * z, r = sqrt(r2);
    double rmin = P[P_RMIN];
    if (fabs(r - rmin) <= 1e-6 * rmin) *marg = 1;
    if (!(r >= rmin)) return 0;
    if (!(rho >= 1e-6 * r)) return 0;
    /* Eq. (spherical projection); azimuth mapped to [0, 2 pi) */
    double phi = atan2(y, x);
    if (phi < 0) phi += TWO_PI;
    double om = asin(z / r);
    /* J^S, all three rows */
    double *J = st->J;
    J[0] = -y / rho2; J[1] = x / rho2; J[2] = 0;
    J[3] = -x * z / (r2 * rho); J[4] = -y * z / (r2 * rho); J[5] = rho / r2;
    J[6] = x / r; J[7] = y / r; J[8] = z / r;
    double cv[6];
    if (!cov2d(st, P[P_LEPS], cv)) return 0;
    double A = cv[0], B = cv[1], C = cv[2], comp = cv[3], det1 = cv[4];
    double op = opac * comp;
    if (fabs(op - ALPHA_MIN) <= 5e-5 * ALPHA_MIN) cull_marg = 1;
    rec[R_MA] = phi; rec[R_MB] = om;
    rec[R_CA] = C / det1; rec[R_CB] = -B / det1; rec[R_CC] = A / det1;
    rec[R_OP] = op;
    rec[R_DEPTH] = r;
    /* v^S = J^S w, three components (Sec. 3.3) */
    for (int i = 0; i < 3; i++) rec[R_VA + i] = J[3 * i] * st->w[0] + J[3 * i + 1] * st->w[1] + J[3 * i + 2] * st->w[2];
    rec[R_SAA] = A; rec[R_SAB] = B; rec[R_SBB] = C;
    rec[R_COMP] = comp;
    /* AABB: k sigma plus the first two components of v^S t_sweep / 2 */
    double half = 0.5 * P[P_SWEEP];
    double k = support_sigmas(P, op);
    rec[R_EXA] = k * sqrt(A) + fabs(rec[R_VA]) * half;
    rec[R_EXB] = k * sqrt(C) + fabs(rec[R_VB]) * half;
    rec[R_LA] = rec[R_HA] = rec[R_EXA];
    rec[R_LB] = rec[R_HB] = rec[R_EXB];
    if ((int)P[P_SUPPORT] & 2) sweep_time_box(P, sqrt(A) * k, sqrt(C) * k, half, rec);
    int nt = lidar_rect(P, elev, rec, 0.0, rect, guard_rad, marg);
    if (cull_marg) *marg = 1;
    if (*marg) {
        int dummy = 0;
        lidar_rect(P, elev, rec, guard_rad, orect, 0.0, &dummy);
        if (!cull_marg) lidar_rect(P, elev, rec, -guard_rad, irect, 0.0, &dummy);
    }
    if (op < ALPHA_MIN) return 0;
    return nt > 0;
}

static int sensor_tiles(const double *P, int *tiles_x, int *tiles_y) {
    if ((int)P[P_KIND] == 0) {
        int tw = (int)P[P_TW], th = (int)P[P_TH];
        *tiles_x = ((int)P[P_WIDTH] + tw - 1) / tw;
        *tiles_y = ((int)P[P_HEIGHT] + th - 1) / th;
    } else {
        *tiles_x = ((int)P[P_NAZ] + (int)P[P_TAZ] - 1) / (int)P[P_TAZ];
        *tiles_y = (int)P[P_NB] / (int)P[P_TEL];
    }
    return *tiles_x * *tiles_y;
}

/* Does the Gaussian's tile rectangle contain tile column tx, row ty? (lidar columns wrap) */
static int rect_contains(const double *P, const int rect[4], int tx, int ty) {
    if (ty < rect[1] || ty >= rect[3]) return 0;
    if ((int)P[P_KIND] == 0) return tx >= rect[0] && tx < rect[2];
    int tiles_x, tiles_y;
    sensor_tiles(P, &tiles_x, &tiles_y);
    int d = ((tx - rect[0]) % tiles_x + tiles_x) % tiles_x;
    return d < rect[2] - rect[0];
}

static int project_one(const double *P, const double *elev, int64_t i, const double *means, const double *scales,
                       const double *quats, const double *opac, const double *vel, proj_state *st, double *rec,
                       int rect[4], int orect[4], int irect[4], double guard, int *marg) {
    if ((int)P[P_KIND] == 0)
        return project_camera(P, means + 3 * i, scales + 3 * i, quats + 4 * i, opac[i], vel ? vel + 3 * i : NULL,
                              st, rec, rect, orect, irect, guard, marg);
    return project_lidar(P, elev, means + 3 * i, scales + 3 * i, quats + 4 * i, opac[i], vel ? vel + 3 * i : NULL,
                         st, rec, rect, orect, irect, guard, marg);
}

/* Public: per-Gaussian projection for one sensor. */
int oracle_project(int64_t n, const double *means, const double *scales, const double *quats, const double *opac,
                   const double *vel, const double *P, const double *elev, double guard, double *rec, int32_t *rect,
                   int32_t *orect, int32_t *irect, int32_t *ntiles, uint8_t *visible, uint8_t *marginal) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        proj_state st;
        int rc[4], orc[4], irc[4], mg;
        int vis = project_one(P, elev, i, means, scales, quats, opac, vel, &st, rec + REC * i, rc, orc, irc, guard, &mg);
        for (int k = 0; k < 4; k++) { rect[4 * i + k] = rc[k]; orect[4 * i + k] = orc[k]; irect[4 * i + k] = irc[k]; }
        ntiles[i] = vis ? (rc[2] - rc[0]) * (rc[3] - rc[1]) : 0;
        visible[i] = (uint8_t)vis;
        marginal[i] = (uint8_t)mg;
    }
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Intersection list of one sensor: all (tile, Gaussian) pairs ordered by tile, then
 * depth, then Gaussian id (Sec. 3.2 tiling and depth sort; Sec. 3.3 range sort).
 * ------------------------------------------------------------------------------- */
typedef struct { int32_t tile; double depth; int32_t id; } isect_t;

static int cmp_isect(const void *a, const void *b) {
    const isect_t *x = (const isect_t *)a, *y = (const isect_t *)b;
    if (x->tile != y->tile) return x->tile < y->tile ? -1 : 1;
    if (x->depth != y->depth) return x->depth < y->depth ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

int64_t oracle_isect_list(int64_t n, const double *P, const double *rec, const int32_t *rect, const int32_t *ntiles,
                          int64_t capacity, int32_t *out_tile, int32_t *out_id) {
    int tiles_x, tiles_y;
    sensor_tiles(P, &tiles_x, &tiles_y);
    int64_t total = 0;
    for (int64_t i = 0; i < n; i++) total += ntiles[i];
    if (total > capacity || !out_tile) return total;
    isect_t *lst = (isect_t *)malloc(sizeof(isect_t) * (size_t)(total > 0 ? total : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++) {
        if (!ntiles[i]) continue;
        const int32_t *rc = rect + 4 * i;
        for (int ty = rc[1]; ty < rc[3]; ty++)
            for (int tx = rc[0]; tx < rc[2]; tx++) {
                int col = ((tx % tiles_x) + tiles_x) % tiles_x;
                if (camera_cull(P) && camera_tile_margin(P, rec + REC * i, col, ty) > 0) continue;
                lst[k].tile = ty * tiles_x + col;
                lst[k].depth = rec[REC * i + R_DEPTH];
                lst[k].id = (int32_t)i;
                k++;
            }
    }
    total = k;
    qsort(lst, (size_t)total, sizeof(isect_t), cmp_isect);
    for (int64_t j = 0; j < total; j++) { out_tile[j] = lst[j].tile; out_id[j] = lst[j].id; }
    free(lst);
    return total;
}

/* Public: the camera tile-cull margins of (tile, Gaussian) query pairs (tile = ty * tiles_x
 * + tx of the sensor), from projected records rec (the option-4 definition above). */
int oracle_tile_margin(const double *P, const double *rec, int64_t nq, const int32_t *tiles, const int32_t *ids,
                       double *out) {
    int tiles_x, tiles_y;
    sensor_tiles(P, &tiles_x, &tiles_y);
    for (int64_t q = 0; q < nq; q++)
        out[q] = camera_tile_margin(P, rec + REC * (int64_t)ids[q], tiles[q] % tiles_x, tiles[q] / tiles_x);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Per-ray blending.
 * ------------------------------------------------------------------------------- */
/* A candidate of a ray: `member` is the Gaussian's tile membership as FP64 decides it;
 * `optional` marks a Gaussian whose membership an FP32 evaluation could decide the
 * other way (its box edge lies within the guard band of a tile edge). */
typedef struct { int32_t id; double depth; int8_t member, optional; } cand_t;

/* Discrete decisions of a ray that lie within the FP32 guard band of their threshold.
 * Each kind is also the ray's bit in the marginal mask. */
enum { D_TILE = 1, D_AMIN = 2, D_AMAX = 4, D_TERM = 8, D_MED = 16, D_TIE = 32, D_LOS = 64, D_RAYTILE = 128 };
typedef struct { int32_t kind, id, id2; } decision_t;

/* Flips to apply (a decision named by kind and Gaussian id is taken the other way) and a
 * recorder of the near decisions met; either part may be empty. */
typedef struct {
    const decision_t *flip;
    int nflip;
    decision_t *near;
    int cap, n_near;
} dec_ctx;

static int flipped(const dec_ctx *dc, int kind, int32_t id) {
    if (!dc) return 0;
    for (int q = 0; q < dc->nflip; q++)
        if (dc->flip[q].kind == kind && dc->flip[q].id == id) return 1;
    return 0;
}

static void note_decision(dec_ctx *dc, int kind, int32_t id, int32_t id2) {
    if (!dc || !dc->near) return;
    if (dc->n_near < dc->cap) {
        dc->near[dc->n_near].kind = kind;
        dc->near[dc->n_near].id = id;
        dc->near[dc->n_near].id2 = id2;
    }
    dc->n_near++;
}

static int cmp_cand(const void *a, const void *b) {
    const cand_t *x = (const cand_t *)a, *y = (const cand_t *)b;
    if (x->depth != y->depth) return x->depth < y->depth ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

typedef struct {           /* one blended Gaussian of a ray, kept for the backward pass */
    int32_t id;
    double alpha, T, G, dx, dy, t, rrs;
    int clamped;
} contrib_t;

/* Lidar tile of a free ray (App. A.2: a lidar point mapped like a Gaussian of zero
 * extent): column floor(phi / w_phi), the row whose elevation boundaries contain omega;
 * -1 outside the beam fan.  *marg is set within FP32 noise of a tile edge. */
static void free_ray_tile(const double *P, const double *elev, double phi, double om, int *tx, int *ty, int *marg) {
    int nb = (int)P[P_NB], naz = (int)P[P_NAZ], taz = (int)P[P_TAZ], tel = (int)P[P_TEL];
    int mphi = (naz + taz - 1) / taz, mw = nb / tel;
    double wphi = taz * P[P_AZRES];
    double bnd[1025];
    elevation_bounds(elev, nb, tel, bnd);
    *tx = *ty = -1;
    for (int k = 0; k <= mw; k++)
        if (fabs(om - bnd[k]) < 2e-7) *marg = 1;
    if (frac_dist(phi / wphi) < 2e-6 || phi < 2e-7 || fabs(phi - TWO_PI) < 2e-7) *marg = 1;
    if (!(om > bnd[0]) || !(om < bnd[mw]) || !(phi >= 0) || !(phi < TWO_PI)) return;
    int c = (int)floor(phi / wphi);
    if (c > mphi - 1) c = mphi - 1;
    int r = 0;
    for (int k = 1; k < mw; k++)
        if (bnd[k] <= om) r = k;
    *tx = c;
    *ty = r;
}

/* Ray geometry: tile, sample point and time.
 *   camera: pixel centre (col+0.5, row+0.5); t_pix = ((row+0.5)/H - 0.5) t_rs + offset (Eq. t_pix)
 *   lidar:  regular grid phi=(a+0.5) res, omega = beam elevation,
 *           t = ((a+0.5)/n_az - 0.5) t_sweep, unless explicit (phi, omega, t) are given. */
static void ray_setup(const double *P, const double *elev, const double *rays, int64_t nfree, int64_t k, int *tx,
                      int *ty, double *pa, double *pb, double *t, int *marg) {
    if (nfree > 0) {   /* free lidar rays (App. A.2): (phi, omega, t) per ray, tile from them */
        *pa = rays[3 * k]; *pb = rays[3 * k + 1]; *t = rays[3 * k + 2];
        free_ray_tile(P, elev, *pa, *pb, tx, ty, marg);
        return;
    }
    if ((int)P[P_KIND] == 0) {
        int W = (int)P[P_WIDTH], H = (int)P[P_HEIGHT];
        int row = (int)(k / W), col = (int)(k % W);
        *tx = col / (int)P[P_TW];
        *ty = row / (int)P[P_TH];
        *pa = col + 0.5;
        *pb = row + 0.5;
        *t = ((row + 0.5) / H - 0.5) * P[P_RS] + P[P_DT];
    } else {
        int naz = (int)P[P_NAZ];
        int b = (int)(k / naz), a = (int)(k % naz);
        *tx = a / (int)P[P_TAZ];
        *ty = b / (int)P[P_TEL];
        if (rays) {
            *pa = rays[3 * k]; *pb = rays[3 * k + 1]; *t = rays[3 * k + 2];
        } else {
            *pa = (a + 0.5) * P[P_AZRES];
            *pb = elev[b];
            *t = ((a + 0.5) / naz - 0.5) * P[P_SWEEP];
        }
    }
}

static double wrap_pi(double d) { return d - TWO_PI * floor((d + M_PI) / TWO_PI); }

/* Candidates of one ray: every visible Gaussian whose tile rectangle holds the ray's
 * tile (every visible Gaussian with P_ALLG), plus the Gaussians whose membership is
 * uncertain in FP32 and that would be blended here, sorted by (depth, id).  Sets bit
 * D_TILE of *mg and records a D_TILE decision for each uncertain one that matters. */
static int gather_candidates(const double *P, int64_t n, const double *rec, const int32_t *rect,
                             const int32_t *orect, const int32_t *irect, const uint8_t *vis, const uint8_t *gmarg,
                             int tx, int ty, double pa, double pb, double t, cand_t *cands, int *mg, dec_ctx *dc) {
    int nc = 0;
    for (int64_t i = 0; i < n; i++) {
        int optional = 0;
        /* a marginal Gaussian's membership is uncertain between its inner and outer boxes;
         * it matters only where it would be blended (alpha at or above the threshold) */
        if (gmarg && gmarg[i] && rect_contains(P, orect + 4 * i, tx, ty) &&
            !rect_contains(P, irect + 4 * i, tx, ty)) {
            const double *g = rec + REC * i;
            double dx = pa - (g[R_MA] + g[R_VA] * t), dy = pb - (g[R_MB] + g[R_VB] * t);
            if ((int)P[P_KIND] == 1) dx = wrap_pi(dx);
            double sig = 0.5 * (g[R_CA] * dx * dx + g[R_CC] * dy * dy) + g[R_CB] * dx * dy;
            if (sig >= 0 && g[R_OP] * exp(-sig) >= ALPHA_MIN * (1 - 1e-4)) {
                *mg |= D_TILE;
                optional = 1;
                note_decision(dc, D_TILE, (int32_t)i, -1);
            }
        }
        int member = vis[i] && (P[P_ALLG] >= 0.5 || rect_contains(P, rect + 4 * i, tx, ty));
        /* the camera tile cull drops pairs that cannot blend anywhere in the tile */
        if (member && P[P_ALLG] < 0.5 && camera_cull(P) && camera_tile_margin(P, rec + REC * i, tx, ty) > 0)
            member = 0;
        if (!member && !optional) continue;
        cands[nc].id = (int32_t)i;
        cands[nc].depth = rec[REC * i + R_DEPTH];
        cands[nc].member = (int8_t)member;
        cands[nc].optional = (int8_t)optional;
        nc++;
    }
    qsort(cands, (size_t)nc, sizeof(cand_t), cmp_cand);
    return nc;
}

/* Front-to-back blend of a ray's sorted candidates (Eq. alpha blend / alpha / delta and
 * the range blend of Sec. 3.3).  Decisions named in dc->flip are taken the other way:
 *   D_TILE: membership of an optional candidate;   D_AMIN: the alpha >= 1/255 test;
 *   D_TERM: the stop before T would fall below 1e-4; D_MED: the T < 1/2 crossing;
 *   D_TIE: the order of two Gaussians blended one after the other (a depth tie);
 *   D_LOS: the line-of-sight cut r_rs < r_p - eps.
 * Decisions within the guard band are recorded in dc and flagged in *mg.  Returns the
 * number of blended Gaussians (written to cb if non-null). */
static int blend_ray(const double *P, const double *rec, const double *feat, int C, const cand_t *cands_in, int nc,
                     double pa, double pb, double t, double *F, double *Tout, double *Dexp, double *Dmed, int *mg,
                     contrib_t *cb, int cb_cap, double rp, double los_eps, double *los, dec_ctx *dc, cand_t *work) {
    int lidar = (int)P[P_KIND] == 1;
    const cand_t *cands = cands_in;
    if (dc && work) {   /* depth ties taken the other way: swap the two Gaussians' places */
        int any = 0;
        for (int q = 0; q < dc->nflip; q++) any |= dc->flip[q].kind == D_TIE;
        if (any) {
            memcpy(work, cands_in, sizeof(cand_t) * (size_t)nc);
            for (int q = 0; q < dc->nflip; q++) {
                if (dc->flip[q].kind != D_TIE) continue;
                int ja = -1, jb = -1;
                for (int j = 0; j < nc; j++) {
                    if (work[j].id == dc->flip[q].id) ja = j;
                    if (work[j].id == dc->flip[q].id2) jb = j;
                }
                if (ja >= 0 && jb >= 0) {
                    cand_t tmp = work[ja];
                    work[ja] = work[jb];
                    work[jb] = tmp;
                }
            }
            cands = work;
        }
    }
    for (int c = 0; c < C; c++) F[c] = 0;
    double T = 1, de = 0, dm = 0, last_depth = -1e300, lsum = 0;
    int med = 0, nb = 0;
    int32_t last_id = -1;
    for (int j = 0; j < nc; j++) {
        const int32_t id = cands[j].id;
        int member = cands[j].member;
        if (cands[j].optional && flipped(dc, D_TILE, id)) member = !member;
        const double *g = rec + REC * id;
        /* Eq. (delta): the mean shifted by the sensor-space velocity at the ray's time */
        double dx = pa - (g[R_MA] + g[R_VA] * t);
        double dy = pb - (g[R_MB] + g[R_VB] * t);
        if (lidar) dx = wrap_pi(dx); /* reading: azimuth difference wrapped to [-pi, pi) */
        double sig = 0.5 * (g[R_CA] * dx * dx + g[R_CC] * dy * dy) + g[R_CB] * dx * dy;
        if (sig < 0) continue;
        double G = exp(-sig);
        double a = g[R_OP] * G;
        int near_min = fabs(a - ALPHA_MIN) <= 5e-5 * ALPHA_MIN;
        /* an optional candidate left out still records its alpha decision: an FP32 run that
         * keeps it (a cull decision near o' = 1/255, then alpha near 1/255 at the centre)
         * takes both */
        if (near_min) { *mg |= D_AMIN; note_decision(dc, D_AMIN, id, -1); }
        if (!member) continue;
        if (fabs(a - ALPHA_MAX) <= 5e-5 * ALPHA_MAX) *mg |= D_AMAX;
        int clamped = 0;
        if (a > ALPHA_MAX) { a = ALPHA_MAX; clamped = 1; }
        int skip = a < ALPHA_MIN;
        if (near_min && flipped(dc, D_AMIN, id)) skip = !skip;
        if (skip) continue;
        /* two blended Gaussians this close in depth may swap order in FP32 */
        if (cands[j].depth - last_depth < 1e-6 * cands[j].depth) {
            *mg |= D_TIE;
            note_decision(dc, D_TIE, last_id, id);
        }
        last_depth = cands[j].depth;
        last_id = id;
        double Tn = T * (1 - a);
        int stop = Tn < T_EPS;
        if (fabs(Tn - T_EPS) <= 2e-3 * T_EPS) {
            *mg |= D_TERM;
            note_decision(dc, D_TERM, id, -1);
            if (flipped(dc, D_TERM, id)) stop = !stop;
        }
        if (stop) break;
        double rrs = g[R_DEPTH] + g[R_VR] * t; /* r_rs = r + v_r t_l */
        const double *f = feat + (int64_t)C * id;
        for (int c = 0; c < C; c++) F[c] += f[c] * a * T;
        de += rrs * a * T;
        int cross = Tn < 0.5;
        if (fabs(Tn - 0.5) <= 1e-3 * 0.5) {
            *mg |= D_MED;
            note_decision(dc, D_MED, id, -1);
            if (flipped(dc, D_MED, id)) cross = !cross;
        }
        if (!med && cross) { dm = rrs; med = 1; }
        /* line-of-sight term (App. B): alpha of every blended Gaussian in front of the
         * return by more than eps; a range within the guard band of the cut is marginal */
        if (los) {
            int front = rrs < rp - los_eps;
            if (fabs(rrs - (rp - los_eps)) <= 1e-5 * fabs(rp)) {
                *mg |= D_LOS;
                note_decision(dc, D_LOS, id, -1);
                if (flipped(dc, D_LOS, id)) front = !front;
            }
            if (front) lsum += a;
        }
        if (cb && nb < cb_cap) {
            contrib_t *e = cb + nb;
            e->id = id; e->alpha = a; e->T = T; e->G = G; e->dx = dx; e->dy = dy; e->t = t;
            e->rrs = rrs; e->clamped = clamped;
        }
        nb++;
        T = Tn;
    }
    *Tout = T;
    if (los) *los = lsum;
    if (Dexp) *Dexp = de;
    if (Dmed) *Dmed = dm;
    return nb;
}

/* Render one ray: returns the number of blended Gaussians (written to cb if non-null). */
static int render_ray(const double *P, const double *elev, const double *rays, int64_t nfree, int64_t n,
                      const double *rec,
                      const int32_t *rect, const int32_t *orect, const int32_t *irect, const uint8_t *vis,
                      const uint8_t *gmarg,
                      const double *feat, int C,
                      int64_t k, cand_t *cands, double *F, double *Tout, double *Dexp, double *Dmed,
                      int *marginal, contrib_t *cb, int cb_cap, double rp, double los_eps, double *los) {
    int tx, ty, tmarg = 0;
    double pa, pb, t;
    ray_setup(P, elev, rays, nfree, k, &tx, &ty, &pa, &pb, &t, &tmarg);
    int mg = tmarg ? D_RAYTILE : 0;
    int nc = gather_candidates(P, n, rec, rect, orect, irect, vis, gmarg, tx, ty, pa, pb, t, cands, &mg, NULL);
    int nb = blend_ray(P, rec, feat, C, cands, nc, pa, pb, t, F, Tout, Dexp, Dmed, &mg, cb, cb_cap, rp, los_eps, los,
                       NULL, NULL);
    if (marginal) *marginal = mg;
    return nb;
}

/* Project every Gaussian; marginal ones (a cull or tile-edge decision within the guard
 * band of FP32 noise) also get an outer rectangle, widened by the guard, that bounds
 * every tile an FP32 evaluation could assign them to. */
static void project_all(int64_t n, const double *means, const double *scales, const double *quats, const double *opac,
                        const double *vel, const double *P, const double *elev, double guard, double *rec,
                        int32_t *rect, int32_t *orect, int32_t *irect, uint8_t *vis, uint8_t *marg) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        proj_state st;
        int rc[4], orc[4], irc[4], mg;
        vis[i] = (uint8_t)project_one(P, elev, i, means, scales, quats, opac, vel, &st, rec + REC * i, rc, orc, irc,
                                      guard, &mg);
        for (int q = 0; q < 4; q++) { rect[4 * i + q] = rc[q]; orect[4 * i + q] = orc[q]; irect[4 * i + q] = irc[q]; }
        marg[i] = (uint8_t)mg;
    }
}

static int64_t sensor_rays(const double *P) {
    if ((int)P[P_KIND] == 0) return (int64_t)P[P_WIDTH] * (int64_t)P[P_HEIGHT];
    return (int64_t)P[P_NB] * (int64_t)P[P_NAZ];
}

/* Public: render the selected rays (sel == NULL: all rays) of one sensor.
 * Outputs per selected ray: F[C], T, expected range, median range, marginal flag,
 * number of blended Gaussians. */
int oracle_render(int64_t n, const double *means, const double *scales, const double *quats, const double *opac,
                  const double *vel, const double *feat, int C, const double *P, const double *elev,
                  const double *rays, int64_t nfree, double guard, int64_t n_sel, const int64_t *sel, double *outF,
                  double *outT,
                  double *outDexp, double *outDmed, uint8_t *outMarg, int32_t *outCount, const double *los_range,
                  double los_eps, double *outLos) {
    double *rec = (double *)malloc(sizeof(double) * REC * (size_t)(n > 0 ? n : 1));
    int32_t *rect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
    int32_t *orect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
    int32_t *irect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
    uint8_t *vis = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    uint8_t *marg = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    project_all(n, means, scales, quats, opac, vel, P, elev, guard, rec, rect, orect, irect, vis, marg);
    int64_t nr = sel ? n_sel : (nfree > 0 ? nfree : sensor_rays(P));
#pragma omp parallel
    {
        cand_t *cands = (cand_t *)malloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t j = 0; j < nr; j++) {
            int64_t k = sel ? sel[j] : j;
            double T, de, dm;
            int mg;
            double lsum = 0;
            int cnt = render_ray(P, elev, rays, nfree, n, rec, rect, orect, irect, vis, marg, feat, C, k, cands,
                                 outF + (int64_t)C * j, &T, &de, &dm, &mg, NULL, 0, los_range ? los_range[j] : 0,
                                 los_eps, los_range ? &lsum : NULL);
            if (outLos) outLos[j] = lsum;
            outT[j] = T;
            if (outDexp) outDexp[j] = de;
            if (outDmed) outDmed[j] = dm;
            if (outMarg) outMarg[j] = (uint8_t)mg;
            if (outCount) outCount[j] = cnt;
        }
        free(cands);
    }
    free(rec); free(rect); free(orect); free(irect); free(vis); free(marg);
    return 0;
}

/* Public: the selected rays rendered under every admissible resolution of their near
 * decisions.  A ray whose FP64 evaluation meets decisions within the guard band of
 * their thresholds (the marginal mask) has more than one result an FP32 evaluation may
 * correctly reach: one per way of taking those decisions.  Variant 0 is the FP64
 * render; variants 1 .. 2^d - 1 take the subsets of the d near decisions the other
 * way (d <= max_dec, 2^max_dec <= max_var).  A ray with more than max_dec near decisions
 * keeps variant 0 only (its outNdec exceeds max_dec: unresolved).
 * Outputs per selected ray j: outF[(j * max_var + v) * C + c], outT / outDexp / outDmed /
 * outLos[j * max_var + v], outNvar[j] variants, outMarg[j] the marginal mask, outNdec[j]
 * the number of near decisions. */
int oracle_render_variants(int64_t n, const double *means, const double *scales, const double *quats,
                           const double *opac, const double *vel, const double *feat, int C, const double *P,
                           const double *elev, const double *rays, int64_t nfree, double guard, int64_t n_sel,
                           const int64_t *sel, const double *los_range, double los_eps, int max_dec, int max_var,
                           double *outF, double *outT, double *outDexp, double *outDmed, double *outLos,
                           int32_t *outNvar, uint8_t *outMarg, int32_t *outNdec) {
    if (max_dec < 0 || max_dec > 16 || (1 << max_dec) > max_var) return -1;
    double *rec = (double *)malloc(sizeof(double) * REC * (size_t)(n > 0 ? n : 1));
    int32_t *rect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
    int32_t *orect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
    int32_t *irect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
    uint8_t *vis = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    uint8_t *marg = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    project_all(n, means, scales, quats, opac, vel, P, elev, guard, rec, rect, orect, irect, vis, marg);
    int64_t nr = sel ? n_sel : (nfree > 0 ? nfree : sensor_rays(P));
#pragma omp parallel
    {
        cand_t *cands = (cand_t *)malloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
        cand_t *work = (cand_t *)malloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
        decision_t near[64], flip[16];
#pragma omp for schedule(dynamic, 16)
        for (int64_t j = 0; j < nr; j++) {
            int64_t k = sel ? sel[j] : j;
            int tx, ty, tmarg = 0;
            double pa, pb, t;
            ray_setup(P, elev, rays, nfree, k, &tx, &ty, &pa, &pb, &t, &tmarg);
            int mg = tmarg ? D_RAYTILE : 0;
            dec_ctx dc = {NULL, 0, near, 64, 0};
            int nc = gather_candidates(P, n, rec, rect, orect, irect, vis, marg, tx, ty, pa, pb, t, cands, &mg, &dc);
            double rp = los_range ? los_range[j] : 0;
            const int64_t o = j * max_var;
            double lsum = 0;
            blend_ray(P, rec, feat, C, cands, nc, pa, pb, t, outF + o * C, outT + o, outDexp ? outDexp + o : NULL,
                      outDmed ? outDmed + o : NULL, &mg, NULL, 0, rp, los_eps, los_range ? &lsum : NULL, &dc, NULL);
            if (outLos) outLos[o] = lsum;
            int nd = dc.n_near;
            int nv = 1;
            if (nd <= max_dec) {
                nv = 1 << nd;
                for (int m = 1; m < nv; m++) {
                    int nf = 0;
                    for (int q = 0; q < nd; q++)
                        if (m & (1 << q)) flip[nf++] = near[q];
                    dec_ctx fc = {flip, nf, NULL, 0, 0};
                    int mg2 = 0;
                    double l2 = 0;
                    blend_ray(P, rec, feat, C, cands, nc, pa, pb, t, outF + (o + m) * C, outT + o + m,
                              outDexp ? outDexp + o + m : NULL, outDmed ? outDmed + o + m : NULL, &mg2, NULL, 0, rp,
                              los_eps, los_range ? &l2 : NULL, &fc, work);
                    if (outLos) outLos[o + m] = l2;
                }
            }
            outNvar[j] = nv;
            outMarg[j] = (uint8_t)mg;
            outNdec[j] = nd;
        }
        free(cands); free(work);
    }
    free(rec); free(rect); free(orect); free(irect); free(vis); free(marg);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Backward of the blend (reverse mode of Eq. alpha blend / alpha / delta and of the
 * range blend), per ray back to front.  Produces per-Gaussian gradients of the
 * projected quantities: d2[10] = (d mean_a, d mean_b, d ca, d cb, d cc, d o',
 * d depth, d va, d vb, d vr), and of the features.
 * ------------------------------------------------------------------------------- */
static void ray_backward(const double *P, int C, const double *feat, const double *rec, const contrib_t *cb, int nb,
                         double Tfinal, const double *gF, double gT, double gD, double gL, double rp, double los_eps,
                         double *d2, double *dfeat, double *dtime) {
    double B[64];
    double BD = 0;
    for (int c = 0; c < C; c++) B[c] = 0;
    for (int j = nb - 1; j >= 0; j--) {
        const contrib_t *e = cb + j;
        const double *g = rec + REC * e->id;
        const double *f = feat + (int64_t)C * e->id;
        double a = e->alpha, T = e->T, w = a * T;
        double dot = 0;
        for (int c = 0; c < C; c++) {
            double dfc = w * gF[c];
#pragma omp atomic
            dfeat[(int64_t)C * e->id + c] += dfc;
            dot += gF[c] * (f[c] - B[c]);
        }
        double dalpha = T * (dot + gD * (e->rrs - BD)) - gT * Tfinal / (1 - a);
        /* line-of-sight term: d/d alpha_i of sum alpha_i over r_rs,i < r_p - eps */
        if (gL != 0 && e->rrs < rp - los_eps) dalpha += gL;
        /* range channel: r_rs = r + v_r t */
        double drrs = gD * w;
        for (int c = 0; c < C; c++) B[c] = f[c] * a + (1 - a) * B[c];
        BD = e->rrs * a + (1 - a) * BD;
        double loc[10] = {0};
        loc[6] = drrs;
        loc[9] = drrs * e->t;
        if (!e->clamped) {
            loc[5] = dalpha * e->G;
            double dsig = -dalpha * a;
            loc[2] = dsig * 0.5 * e->dx * e->dx;
            loc[3] = dsig * e->dx * e->dy;
            loc[4] = dsig * 0.5 * e->dy * e->dy;
            double ddx = dsig * (g[R_CA] * e->dx + g[R_CB] * e->dy);
            double ddy = dsig * (g[R_CB] * e->dx + g[R_CC] * e->dy);
            loc[0] = -ddx; loc[1] = -ddy;
            loc[7] = -ddx * e->t; loc[8] = -ddy * e->t;
            /* the ray time (row time + camera time offset) moves the mean by v t */
            if (dtime) *dtime += -(ddx * g[R_VA] + ddy * g[R_VB]);
        }
        for (int q = 0; q < 10; q++) {
#pragma omp atomic
            d2[10 * e->id + q] += loc[q];
        }
    }
    (void)P;
}

/* d conic (as stored: a, b, c with matrix [[a,b],[b,c]]) -> d (A, B, C) of Sigma'=[[A,B],[B,C]]
 * by differentiating conic = [C, -B, A] / (AC - B^2) parameter by parameter. */
static void conic_backward(double A, double B, double C, const double dcon[3], double dS[3]) {
    double D = A * C - B * B, D2 = D * D;
    double dca_dA = -C * C / D2, dca_dB = 2 * B * C / D2, dca_dC = 1 / D - C * A / D2;
    double dcb_dA = B * C / D2, dcb_dB = -1 / D - 2 * B * B / D2, dcb_dC = B * A / D2;
    double dcc_dA = 1 / D - A * C / D2, dcc_dB = 2 * A * B / D2, dcc_dC = -A * A / D2;
    dS[0] = dcon[0] * dca_dA + dcon[1] * dcb_dA + dcon[2] * dcc_dA;
    dS[1] = dcon[0] * dca_dB + dcon[1] * dcb_dB + dcon[2] * dcc_dB;
    dS[2] = dcon[0] * dca_dC + dcon[1] * dcb_dC + dcon[2] * dcc_dC;
}

/* Partial derivatives of R(q) entries with respect to the normalised quaternion. */
static void dR_dq(const double q[4], double d[4][9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    double dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    double dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    double dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    memcpy(d[0], dw, sizeof dw); memcpy(d[1], dx, sizeof dx);
    memcpy(d[2], dy, sizeof dy); memcpy(d[3], dz, sizeof dz);
}

/* Partial derivatives of the 9 entries of J (camera rows 0,1 or lidar J^S) w.r.t. the
 * sensor-frame mean (x, y, z): dJ[e][k] = d J_e / d m_k. */
static void dJ_dm(const double *P, const proj_state *st, double dJ[9][3]) {
    memset(dJ, 0, sizeof(double) * 27);
    double x = st->m[0], y = st->m[1], z = st->m[2];
    if ((int)P[P_KIND] == 0) {
        double fx = P[P_FX], fy = P[P_FY];
        dJ[0][2] = -fx / (z * z);
        dJ[4][2] = -fy / (z * z);
        /* J02 = -fx tx / z^2 with tx = x (free) or z*L (clamped) */
        if (!st->clamp_x) { dJ[2][0] = -fx / (z * z); dJ[2][2] = 2 * fx * x / (z * z * z); }
        else { double L = clampd(x / z, -st->lim_x, st->lim_x); dJ[2][2] = fx * L / (z * z); }
        if (!st->clamp_y) { dJ[5][1] = -fy / (z * z); dJ[5][2] = 2 * fy * y / (z * z * z); }
        else { double L = clampd(y / z, -st->lim_y, st->lim_y); dJ[5][2] = fy * L / (z * z); }
        return;
    }
    double rho2 = x * x + y * y, rho = sqrt(rho2), r2 = rho2 + z * z, r = sqrt(r2);
    double rho4 = rho2 * rho2;
    /* row 0: -y/rho^2, x/rho^2, 0 */
    dJ[0][0] = 2 * x * y / rho4; dJ[0][1] = (y * y - x * x) / rho4;
    dJ[1][0] = (y * y - x * x) / rho4; dJ[1][1] = -2 * x * y / rho4;
    /* row 1: -xz/h, -yz/h, rho/r^2 with h = r^2 rho */
    double h = r2 * rho, h2 = h * h;
    double dh[3] = {2 * x * rho + r2 * x / rho, 2 * y * rho + r2 * y / rho, 2 * z * rho};
    dJ[3][0] = -z / h + x * z * dh[0] / h2; dJ[3][1] = x * z * dh[1] / h2; dJ[3][2] = -x / h + x * z * dh[2] / h2;
    dJ[4][0] = y * z * dh[0] / h2; dJ[4][1] = -z / h + y * z * dh[1] / h2; dJ[4][2] = -y / h + y * z * dh[2] / h2;
    double r4 = r2 * r2;
    dJ[5][0] = (x / rho) / r2 - 2 * x * rho / r4;
    dJ[5][1] = (y / rho) / r2 - 2 * y * rho / r4;
    dJ[5][2] = -2 * z * rho / r4;
    /* row 2: m/r */
    double r3 = r2 * r;
    double m[3] = {x, y, z};
    for (int a = 0; a < 3; a++)
        for (int k = 0; k < 3; k++) dJ[6 + a][k] = (a == k ? 1 / r : 0) - m[a] * m[k] / r3;
}

/* Chain rule from projected-quantity gradients d2[10] to the Gaussian parameters. */
static void projection_backward(const double *P, const double *elev, int64_t i, const double *means,
                                const double *scales, const double *quats, const double *opac, const double *vel,
                                const double *d2, double *dmean, double *dscale, double *dquat, double *dopac,
                                double *dvel, double *dsensor) {
    proj_state st;
    double rec[REC];
    int rc[4], orc[4], irc[4], mg;
    if (!project_one(P, elev, i, means, scales, quats, opac, vel, &st, rec, rc, orc, irc, 0.0, &mg)) return;
    int lidar = (int)P[P_KIND] == 1;
    const double *J = st.J;
    double dm[3] = {0, 0, 0};
    double dJ[9] = {0};
    /* 2-D mean */
    if (!lidar) {
        double x = st.m[0], y = st.m[1], z = st.m[2];
        double dux = P[P_FX] * d2[0], duy = P[P_FY] * d2[1];
        dm[0] += dux / z; dm[1] += duy / z; dm[2] += -dux * x / (z * z) - duy * y / (z * z);
    } else {
        double ds[3] = {d2[0], d2[1], d2[6]}; /* (phi, omega, r) */
        for (int k = 0; k < 3; k++) dm[k] += J[k] * ds[0] + J[3 + k] * ds[1] + J[6 + k] * ds[2];
    }
    /* conic and compensation -> Sigma_2d entries (a, b, c) */
    double A = rec[R_SAA], B = rec[R_SAB], C = rec[R_SBB];
    double eps = lidar ? P[P_LEPS] : P[P_EPS];
    double dcon[3] = {d2[2], d2[3], d2[4]}, dS[3];
    conic_backward(A, B, C, dcon, dS);
    double a = A - eps, c = C - eps, b = B;
    double det0 = a * c - b * b, det1 = A * C - B * B, comp = rec[R_COMP];
    dopac[i] += d2[5] * comp;
    double dcomp = d2[5] * opac[i];
    if (det0 > 0 && comp > 0) {
        double dq = dcomp / (2 * comp), D2 = det1 * det1;
        dS[0] += dq * (c * det1 - det0 * C) / D2;
        dS[2] += dq * (a * det1 - det0 * A) / D2;
        dS[1] += dq * (-2 * b * det1 + 2 * b * det0) / D2;
    }
    /* Sigma_2d = J2 Sc J2^T */
    double Sc[9];
    memcpy(Sc, st.Sc, sizeof Sc);
    double dSc[9];
    for (int p = 0; p < 3; p++)
        for (int q = 0; q < 3; q++)
            dSc[3 * p + q] = dS[0] * J[p] * J[q] + dS[1] * J[p] * J[3 + q] + dS[2] * J[3 + p] * J[3 + q];
    for (int p = 0; p < 3; p++) {
        double s0 = 0, s1 = 0;
        for (int q = 0; q < 3; q++) { s0 += Sc[3 * p + q] * J[q]; s1 += Sc[3 * p + q] * J[3 + q]; }
        dJ[p] += 2 * dS[0] * s0 + dS[1] * s1;
        dJ[3 + p] += dS[1] * s0 + 2 * dS[2] * s1;
    }
    /* velocity v = J w (2 rows camera, 3 rows lidar) */
    int nrow = lidar ? 3 : 2;
    double dv[3] = {d2[7], d2[8], lidar ? d2[9] : 0};
    double dw[3] = {0, 0, 0};
    for (int rr = 0; rr < nrow; rr++)
        for (int k = 0; k < 3; k++) { dJ[3 * rr + k] += dv[rr] * st.w[k]; dw[k] += J[3 * rr + k] * dv[rr]; }
    /* J(m) */
    double dJm[9][3];
    dJ_dm(P, &st, dJm);
    for (int e = 0; e < 9; e++)
        for (int k = 0; k < 3; k++) dm[k] += dJ[e] * dJm[e][k];
    /* w = -omega x m - v_s + R v_g */
    double oxdw[3];
    cross3(P + P_W, dw, oxdw);
    for (int k = 0; k < 3; k++) dm[k] += oxdw[k];
    /* sensor velocities (the paper optimises both): dL/dv_s = -dL/dw, dL/domega = dL/dw x m */
    if (dsensor) {
        double dwxm[3];
        cross3(dw, st.m, dwxm);
        for (int k = 0; k < 3; k++) {
#pragma omp atomic
            dsensor[k] -= dw[k];
#pragma omp atomic
            dsensor[3 + k] += dwxm[k];
        }
    }
    /* sensor pose: m = R mu + t, Sc = R S R^T, w contains R v_g.  Translation: dL/dt = dm.
     * Rotation, perturbed as R <- (I + [theta]x) R: the mean moves by theta x (m - t),
     * R v_g by theta x (R v_g), and Sc by [theta]x Sc - Sc [theta]x, whose gradient is
     * 2 axial(Sc G - G Sc) with G = dL/dSc. */
    if (dsensor) {
        double a[3], rv[3], c1[3], c2[3];
        const double *Rm = P + P_R, *tt = P + P_T;
        for (int k = 0; k < 3; k++) {
            a[k] = st.m[k] - tt[k];
            rv[k] = vel ? Rm[3 * k] * vel[3 * i] + Rm[3 * k + 1] * vel[3 * i + 1] + Rm[3 * k + 2] * vel[3 * i + 2] : 0;
        }
        cross3(a, dm, c1);
        cross3(rv, dw, c2);
        double Gs[9], M[9];   /* Sc G with G the symmetric part of dL/dSc (Sc is symmetric) */
        for (int p = 0; p < 3; p++)
            for (int q = 0; q < 3; q++) Gs[3 * p + q] = 0.5 * (dSc[3 * p + q] + dSc[3 * q + p]);
        mm3(st.Sc, Gs, M);
        const double ax[3] = {2 * (M[5] - M[7]), 2 * (M[6] - M[2]), 2 * (M[1] - M[3])};
        for (int k = 0; k < 3; k++) {
#pragma omp atomic
            dsensor[8 + k] += dm[k];
#pragma omp atomic
            dsensor[11 + k] += c1[k] + c2[k] + ax[k];
        }
    }
    const double *R = P + P_R;
    if (dvel)
        for (int k = 0; k < 3; k++) dvel[3 * i + k] += R[k] * dw[0] + R[3 + k] * dw[1] + R[6 + k] * dw[2];
    for (int k = 0; k < 3; k++) dmean[3 * i + k] += R[k] * dm[0] + R[3 + k] * dm[1] + R[6 + k] * dm[2];
    /* Sc = R S R^T -> dS_world = R^T dSc R */
    double tmp[9], dSw[9];
    mtm3(R, dSc, tmp);
    mm3(tmp, R, dSw);
    /* S = M M^T with M = Rq diag(s) */
    double M[9], dM[9], sym[9];
    for (int p = 0; p < 3; p++)
        for (int q = 0; q < 3; q++) { M[3 * p + q] = st.Rq[3 * p + q] * st.s[q]; sym[3 * p + q] = dSw[3 * p + q] + dSw[3 * q + p]; }
    mm3(sym, M, dM);
    double dRq[9];
    for (int p = 0; p < 3; p++)
        for (int q = 0; q < 3; q++) {
            dscale[3 * i + q] += dM[3 * p + q] * st.Rq[3 * p + q];
            dRq[3 * p + q] = dM[3 * p + q] * st.s[q];
        }
    double qh[4], dqh[4] = {0, 0, 0, 0}, dR[4][9];
    for (int k = 0; k < 4; k++) qh[k] = st.q[k] / st.qn;
    dR_dq(qh, dR);
    for (int k = 0; k < 4; k++)
        for (int e = 0; e < 9; e++) dqh[k] += dRq[e] * dR[k][e];
    double dot = qh[0] * dqh[0] + qh[1] * dqh[1] + qh[2] * dqh[2] + qh[3] * dqh[3];
    for (int k = 0; k < 4; k++) dquat[4 * i + k] += (dqh[k] - qh[k] * dot) / st.qn;
}

/* Public: full backward for one sensor over the selected rays (sel == NULL: all rays).
 * Upstream gradients, one entry per selected ray:
 * gF[nrays][C], gT[nrays] (d/d final transmittance), gD[nrays] (expected range, lidar
 * only, may be NULL), gA[nrays] (accumulated alpha = 1 - T, lidar, may be NULL).
 * Accumulates (+=) into d2 (n x 10, projected-quantity gradients), dfeat and the
 * parameter gradients. */
int oracle_render_backward(int64_t n, const double *means, const double *scales, const double *quats,
                           const double *opac, const double *vel, const double *feat, int C, const double *P,
                           const double *elev, const double *rays, int64_t nfree, int64_t n_sel, const int64_t *sel,
                           const double *gF, const double *gT, const double *gD, const double *gA, double *d2,
                           double *dfeat, double *dmean, double *dscale, double *dquat, double *dopac, double *dvel,
                           const double *los_range, double los_eps, const double *gL, double *dsensor) {
    if (C > 64) return -1;
    double *rec = (double *)malloc(sizeof(double) * REC * (size_t)(n > 0 ? n : 1));
    int32_t *rect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
    int32_t *orect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
    int32_t *irect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(n > 0 ? n : 1));
    uint8_t *vis = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    uint8_t *marg = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    project_all(n, means, scales, quats, opac, vel, P, elev, 0.0, rec, rect, orect, irect, vis, marg);
    int64_t nr = sel ? n_sel : (nfree > 0 ? nfree : sensor_rays(P));
    double *loc2 = (double *)calloc((size_t)(n > 0 ? n : 1) * 10, sizeof(double));
#pragma omp parallel
    {
        cand_t *cands = (cand_t *)malloc(sizeof(cand_t) * (size_t)(n > 0 ? n : 1));
        contrib_t *cb = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)(n > 0 ? n : 1));
        double F[64];
#pragma omp for schedule(dynamic, 16)
        for (int64_t j = 0; j < nr; j++) {
            const int64_t k = sel ? sel[j] : j;   /* ray index; upstream gradients are indexed by j */
            double T, de, dm;
            int nb = render_ray(P, elev, rays, nfree, n, rec, rect, orect, irect, vis, NULL, feat, C, k, cands, F, &T, &de,
                                &dm,
                                NULL, cb, (int)(n > 0 ? n : 1), 0, 0, NULL);
            double gt = gT ? gT[j] : 0;
            if (gA) gt -= gA[j]; /* alpha_acc = 1 - T */
            double dt = 0;
            ray_backward(P, C, feat, rec, cb, nb, T, gF + (int64_t)C * j, gt, gD ? gD[j] : 0,
                         (gL && los_range) ? gL[j] : 0, los_range ? los_range[j] : 0, los_eps, loc2, dfeat,
                         (dsensor && (int)P[P_KIND] == 0) ? &dt : NULL);
            if (dsensor) {
#pragma omp atomic
                dsensor[6] += dt;
            }
        }
        free(cands); free(cb);
    }
    for (int64_t i = 0; i < n * 10; i++) d2[i] += loc2[i];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        if (!vis[i]) continue;
        projection_backward(P, elev, i, means, scales, quats, opac, vel, loc2 + 10 * i, dmean, dscale, dquat, dopac,
                            dvel, dsensor);
    }
    free(loc2); free(rec); free(rect); free(orect); free(irect); free(vis); free(marg);
    return 0;
}

/* Public: chain rule only (for tests that feed their own projected-quantity gradients). */
int oracle_projection_backward(int64_t n, const double *means, const double *scales, const double *quats,
                               const double *opac, const double *vel, const double *P, const double *elev,
                               const double *d2, double *dmean, double *dscale, double *dquat, double *dopac,
                               double *dvel, double *dsensor) {
    for (int64_t i = 0; i < n; i++)
        projection_backward(P, elev, i, means, scales, quats, opac, vel, d2 + 10 * i, dmean, dscale, dquat, dopac,
                            dvel, dsensor);
    return 0;
}

/* Public: the sensor-space Jacobian rows the projection used (tests compare them with
 * finite differences of the plain projection maps).  J out: 9 doubles. */
int oracle_jacobian(const double *mean, const double *scale, const double *quat, double opac, const double *P,
                    const double *elev, double *J, double *Sc, double *w) {
    proj_state st;
    double rec[REC];
    int rc[4], orc[4], irc[4], mg;
    int vis;
    if ((int)P[P_KIND] == 0)
        vis = project_camera(P, mean, scale, quat, opac, NULL, &st, rec, rc, orc, irc, 0.0, &mg);
    else
        vis = project_lidar(P, elev, mean, scale, quat, opac, NULL, &st, rec, rc, orc, irc, 0.0, &mg);
    memcpy(J, st.J, sizeof(double) * 9);
    memcpy(Sc, st.Sc, sizeof(double) * 9);
    memcpy(w, st.w, sizeof(double) * 3);
    return vis;
}
