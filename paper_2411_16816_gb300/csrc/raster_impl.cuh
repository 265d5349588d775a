// raster_impl.cuh -- tile rasterization of cameras and lidars, forward and backward.
//
// Camera (paper Sec. 3.2 "Rasterization"): one CTA per tile, row time
// t_pix = ((row + 0.5) / H - 0.5) t_rs (+ time offset) (Eq. t_pix), Gaussians blended front
// to back (Eq. alpha blend) with the EWA-blurred alpha of Eq. (alpha) at the rolling-
// shutter shifted mean of Eq. (delta).
// Lidar (Sec. 3.3 "Rasterization", App. A.2): one CTA per lidar tile (N_phi azimuth bins x
// N_omega beams), each ray with its own (phi, omega, t); the expected range blends
// r + v_r t and the median range is the rolling-shutter range of the first Gaussian
// after which the transmittance is below 0.5.  Slots without a ray (the ragged last
// azimuth column) only help stage Gaussians, as in App. A.2.
//
// Each thread owns PX rays of the tile (rays t, t + NT, ... for NT = tile / PX threads),
// so one shared-memory read of a Gaussian serves PX rays and, in the backward, one warp
// reduction of a Gaussian's gradient covers 32 * PX rays.  Gaussians are staged through
// shared memory a tile-sized batch at a time and the block stops once every ray is done
// (__syncthreads_count vote).  The backward walks the list back to front, rebuilding the
// transmittance by division, evaluates each (ray, Gaussian) term branch-free (a ray that
// does not blend the Gaussian gets alpha = 0, which zeroes every term), sums the terms
// over the warp with one transpose reduction, over the CTA in shared memory, and issues
// one set of vector atomics per (tile, Gaussian).  With `out_T`/`out_last` absent it first
// recomputes them for its tile (no per-ray forward state kept).
#pragma once
#include "status.cuh"
#include "types.cuh"

namespace splat {

// Rays per thread.  The camera backward takes four rays per thread for up to 16 channels
// (two for the lidar), so one warp reduction of a Gaussian's gradient covers 128 (64)
// rays; the camera forward takes two (evaluated as a packed pair), the lidar forward one
// (its rays terminate early and it needs the occupancy); wide channel counts keep one ray
// per thread for register room.  A block always keeps at least one full warp.
template <int CM, bool BWD, bool LIDAR, int RAYS>
struct RaysPerThread {
    static constexpr int want = (BWD && CM <= 16) ? (LIDAR ? 2 : 4) : ((!BWD && !LIDAR && CM <= 16) ? 2 : 1);
    static constexpr int value = want * 32 <= RAYS ? want : (2 * 32 <= RAYS ? 2 : 1);
};

struct RayCtx {
    bool inside;
    float pa, pb, t;
    int64_t o;      // output index
};

struct TileCtx {
    int s;          // sensor
    int gtile;      // global tile id
    int tx, ty;     // tile coordinates
};

// Checked-build sites (the status word records the first failing one).
enum : uint32_t {
    kSiteRange = 1,        // a tile range outside [0, *n_isect] (or a non-empty one with n = 0)
    kSiteGaussId = 2,      // a listed Gaussian index >= n
    kSiteRayRange = 3,     // a free-ray list range outside [0, n_rays]
    kSiteRayId = 4,        // a listed ray index >= n_rays
};

// The tile's entry range.  Checked build: a range that does not fit the list is skipped
// (read as empty).
__device__ __forceinline__ int2 load_range(const RasterIn& in, int64_t gtile) {
    int2 r = in.ranges[gtile];
#ifdef SPLAT_CHECKED
    const int64_t len = in.n_isect ? *in.n_isect : 0;
    if (SPLAT_OUT_OF_BOUNDS(r.x == r.y || (in.n > 0 && r.x >= 0 && r.x <= r.y && (int64_t)r.y <= len), kSiteRange))
        r = make_int2(0, 0);
#endif
    return r;
}

// A listed Gaussian index.  Checked build: one past the Gaussians is replaced by 0 (the
// ranges that reach here are non-empty, so n > 0).
__device__ __forceinline__ uint32_t load_id(const RasterIn& in, int64_t j) {
    uint32_t id = in.ids[j];
    if (SPLAT_OUT_OF_BOUNDS((int64_t)id < in.n, kSiteGaussId)) id = 0;
    return id;
}

template <bool LIDAR>
__device__ __forceinline__ TileCtx tile_setup(const Frame& fr) {
    TileCtx c;
    c.s = sensor_of_block(fr, blockIdx.x, LIDAR);
    const SensorDev& S = fr.s[c.s];
    const int lt = blockIdx.x - S.block_base;
    c.tx = lt % S.tiles_x;
    c.ty = lt / S.tiles_x;
    c.gtile = S.tile_base + lt;
    return c;
}

// Ray `p` of tile (tx, ty) for a tile of tw x th rays (runtime shape).
template <bool LIDAR>
__device__ __forceinline__ RayCtx ray_setup_rt(const SensorDev& S, int tx, int ty, int p, int tw, int th) {
    RayCtx r;
    const int lx = p % tw, ly = p / tw;
    if (!LIDAR) {
        const int col = tx * tw + lx, row = ty * th + ly;
        r.inside = col < S.width && row < S.height;
        r.pa = col + 0.5f;
        r.pb = row + 0.5f;
        r.t = ((row + 0.5f) / (float)S.height - 0.5f) * S.rs + S.dt;
        r.o = (int64_t)S.ray_base + (int64_t)row * S.width + col;
    } else {
        const int a = tx * tw + lx, b = ty * th + ly;
        r.inside = a < S.naz;
        r.o = (int64_t)S.ray_base + (int64_t)b * S.naz + a;
        if (r.inside) {
            if (S.rays) {
                const int64_t k = ((int64_t)b * S.naz + a) * 3;
                r.pa = S.rays[k];
                r.pb = S.rays[k + 1];
                r.t = S.rays[k + 2];
            } else {
                r.pa = (a + 0.5f) * S.az_res;
                r.pb = S.elev[b];
                r.t = ((a + 0.5f) / (float)S.naz - 0.5f) * S.sweep;
            }
        } else {
            r.pa = r.pb = r.t = 0.f;
        }
    }
    return r;
}

template <int TW, int TH, bool LIDAR>
__device__ __forceinline__ RayCtx ray_setup(const Frame& fr, const TileCtx& tc, int p /* ray slot in tile */) {
    return ray_setup_rt<LIDAR>(fr.s[tc.s], tc.tx, tc.ty, p, TW, TH);
}

// Block -> (tile, chunk) of a free-ray list: the tile is the last one whose first chunk is
// at or before this block's (tiles without rays own no chunk), the chunk's rays are
// [first, min(first + kListChunk, end)) of ids.  False for the blocks past the last chunk
// (the grid is sized by an upper bound); the whole block returns together.
__device__ __forceinline__ bool list_setup(const Frame& fr, const RayList& L, TileCtx& tc, int& first, int& end) {
    const int chunk = blockIdx.x;
    if (chunk >= L.chunk_base[L.tiles]) return false;
    int lo = 0, hi = L.tiles - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.chunk_base[mid] <= chunk) lo = mid;
        else hi = mid - 1;
    }
    const SensorDev& S = fr.s[L.sensor];
    tc.s = L.sensor;
    tc.gtile = S.tile_base + lo;
    tc.tx = lo % S.tiles_x;
    tc.ty = lo / S.tiles_x;
    int2 rr = L.ranges[lo];
    if (SPLAT_OUT_OF_BOUNDS(rr.x >= 0 && rr.x <= rr.y && (int64_t)rr.y <= L.n_rays, kSiteRayRange))
        rr = make_int2(0, 0);
    first = rr.x + (chunk - L.chunk_base[lo]) * kListChunk;
    end = rr.y;
    return true;
}

// Slot j of the list: its ray (phi, omega, t) and output index (the ray's own index).
__device__ __forceinline__ RayCtx list_ray(const RayList& L, int j, int end) {
    RayCtx r;
    r.inside = j < end;
    r.o = 0;
    r.pa = r.pb = r.t = 0.f;
    if (r.inside) {
        r.o = L.ids[j];
        if (SPLAT_OUT_OF_BOUNDS(r.o >= 0 && r.o < L.n_rays, kSiteRayId)) {
            r.inside = false;
            r.o = 0;
            return r;
        }
        const float* p = L.rays + 3 * r.o;
        r.pa = p[0];
        r.pb = p[1];
        r.t = p[2];
    }
    return r;
}

// The block's tile and this thread's rays: the sensor's ray grid, or a chunk of a free-ray
// list (LIST).  False: a list block without a chunk.
template <int TW, int TH, bool LIDAR, bool LIST, int PX, int NT>
__device__ __forceinline__ bool block_setup(const Frame& fr, const RasterIn& in, TileCtx& tc, RayCtx (&r)[PX]) {
    if constexpr (LIST) {
        static_assert(LIDAR && TW * TH == kListChunk, "list kernels take one chunk of lidar rays per block");
        int first, end;
        if (!list_setup(fr, in.list, tc, first, end)) return false;
#pragma unroll
        for (int q = 0; q < PX; q++) r[q] = list_ray(in.list, first + (int)threadIdx.x + q * NT, end);
    } else {
        tc = tile_setup<LIDAR>(fr);
#pragma unroll
        for (int q = 0; q < PX; q++) r[q] = ray_setup<TW, TH, LIDAR>(fr, tc, threadIdx.x + q * NT);
    }
    return true;
}

template <int CM, int B, bool LIDAR>
struct Stage {
    static_assert(CM % 4 == 0, "features are staged and read as float4");
    float4 g0[B];
    float4 g1[B];
    float2 g2[LIDAR ? B : 1];
    uint32_t id[B];
    // camera: the Gaussian can reach alpha >= 1/255 somewhere in this tile (backward
    // staging); the forward stages only such entries and keeps their list positions here
    int live[LIDAR ? 1 : B];
    alignas(16) float f[B * CM];
};

// Pixel-centre rectangle of a camera tile (clipped to the image) and its row-time range.
struct TileBox {
    float x0, x1, y0, y1, t0, t1;
};

__device__ __forceinline__ TileBox camera_tile_box(const SensorDev& S, int tx, int ty, int tw, int th) {
    TileBox b;
    const int c1 = min(tx * tw + tw, S.width) - 1, r1 = min(ty * th + th, S.height) - 1;
    b.x0 = tx * tw + 0.5f;
    b.x1 = c1 + 0.5f;
    b.y0 = ty * th + 0.5f;
    b.y1 = r1 + 0.5f;
    b.t0 = ((ty * th + 0.5f) / (float)S.height - 0.5f) * S.rs + S.dt;
    b.t1 = ((r1 + 0.5f) / (float)S.height - 0.5f) * S.rs + S.dt;
    return b;
}

// Can the Gaussian reach alpha >= 1/255 at some pixel centre of the tile, at that pixel's
// row time?  alpha >= 1/255 needs d^T K d <= 2 ln(255 o') (K the conic).  The mean moves by
// v t; relative to the mean at mid-time, a pixel at time t acts as a pixel displaced by at
// most |v| (t1 - t0) / 2, so the test grows the rectangle by that sweep and takes the
// minimum of the quadratic form over it (centre inside, else the minimum along an edge).
// Conservative by a small margin: it never calls a tile dead where an FP32 evaluation
// could still blend the Gaussian.
__device__ __forceinline__ bool tile_live(const float4 g0, const float4 g1, const TileBox& b) {
    const float a = g1.x, bb = g1.y, c = g1.z;
    const float thr = 2.f * logf(255.f * g1.w) * 1.001f + 1e-3f;
    if (!(thr >= 0.f)) return false;
    const float tm = 0.5f * (b.t0 + b.t1), ht = 0.5f * fabsf(b.t1 - b.t0);
    const float cx = g0.x + g0.z * tm, cy = g0.y + g0.w * tm;
    const float gx = fabsf(g0.z) * ht + 1e-3f, gy = fabsf(g0.w) * ht + 1e-3f;
    const float u0 = b.x0 - gx - cx, u1 = b.x1 + gx - cx;
    const float v0 = b.y0 - gy - cy, v1 = b.y1 + gy - cy;
    if (u0 <= 0.f && u1 >= 0.f && v0 <= 0.f && v1 >= 0.f) return true;
    auto q = [&](float u, float v) { return a * u * u + 2.f * bb * u * v + c * v * v; };
    auto edge_u = [&](float u) {   // u fixed, v in [v0, v1]
        const float v = fminf(fmaxf(-bb * u / c, v0), v1);
        return q(u, v);
    };
    auto edge_v = [&](float v) {   // v fixed, u in [u0, u1]
        const float u = fminf(fmaxf(-bb * v / a, u0), u1);
        return q(u, v);
    };
    const float m = fminf(fminf(edge_u(u0), edge_u(u1)), fminf(edge_v(v0), edge_v(v1)));
    return !(m > thr);
}

// HALF stages the conic as (a/2, b, c/2, o') for the forward's evaluation.
template <int CM, int B, bool LIDAR, bool HALF = false>
__device__ __forceinline__ void stage_load(Stage<CM, B, LIDAR>& sm, const RasterIn& in, int s, int64_t j, int slot,
                                           const TileBox& box) {
    const uint32_t id = load_id(in, j);
    sm.id[slot] = id;
    const float4 g0 = in.rec[rec_index(s, 0, in.n, id)];
    const float4 g1 = in.rec[rec_index(s, 1, in.n, id)];
    sm.g0[slot] = g0;
    sm.g1[slot] = HALF ? make_float4(__fmul_rn(0.5f, g1.x), g1.y, __fmul_rn(0.5f, g1.z), g1.w) : g1;
    if (!LIDAR) sm.live[slot] = tile_live(g0, g1, box);
    if (LIDAR) {
        const float4 r2 = in.rec[rec_index(s, 2, in.n, id)];
        sm.g2[slot] = make_float2(r2.x, r2.y);
    }
    const int C = in.C;
    const float* fp = in.feat + (int64_t)id * C;
    if ((C & 3) == 0) {
#pragma unroll
        for (int c = 0; c < CM; c += 4) {
            if (c < C) {
                const float4 v = *reinterpret_cast<const float4*>(fp + c);
                *reinterpret_cast<float4*>(&sm.f[slot * CM + c]) = v;
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < CM; c++)
            if (c < C) sm.f[slot * CM + c] = fp[c];
    }
}

// Hardware reciprocal (at most 1 ulp from the rounded result).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// exp(x) as 2^(x log2 e) on the hardware base-2 exponential (ex2.approx, at most 2 ulp).
__device__ __forceinline__ float exp2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
constexpr float kNegLog2e = -1.4426950408889634f;

// alpha of one staged Gaussian at the ray; returns false if it is skipped.  Every step is
// an explicitly rounded operation, in the order eval_alpha2 takes lane by lane, so the
// single-ray and the paired evaluation give the same bits (the forward and the backward
// then agree on every decision):
//   d = p - (mean + v t),  sigma = d_x (a/2 d_x + b d_y) + (c/2 d_y) d_y,
//   alpha = min(o' exp(-sigma), 0.999), blended if sigma >= 0 and alpha >= 1/255.
// HALF: the staged record already holds a/2 and c/2 (the halving is exact, so both forms
// give the same bits).
template <bool LIDAR, bool HALF = false>
__device__ __forceinline__ bool eval_alpha(const float4 g0, const float4 g1, const RayCtx& r, float& dx, float& dy,
                                           float& G, float& alpha, bool& clamped) {
    dx = __fsub_rn(r.pa, __fmaf_rn(g0.z, r.t, g0.x));
    dy = __fsub_rn(r.pb, __fmaf_rn(g0.w, r.t, g0.y));
    if (LIDAR) dx = wrap_pi(dx);
    const float ha = HALF ? g1.x : __fmul_rn(0.5f, g1.x), hc = HALF ? g1.z : __fmul_rn(0.5f, g1.z);
    const float u = __fmaf_rn(ha, dx, __fmul_rn(g1.y, dy));
    const float sig = __fmaf_rn(dx, u, __fmul_rn(__fmul_rn(hc, dy), dy));
    G = exp2_approx(__fmul_rn(sig, kNegLog2e));
    const float a = __fmul_rn(g1.w, G);
    clamped = a > kAlphaMax;
    alpha = clamped ? kAlphaMax : a;
    return sig >= 0.f && alpha >= kAlphaMin;
}

// Two rays of one thread against one staged Gaussian in packed FP32 pairs; lane q equals
// eval_alpha for ray q bit for bit.  pa, pb, t hold the two rays' coordinates and times.
template <bool LIDAR, bool HALF = false>
__device__ __forceinline__ void eval_alpha2(const float4 g0, const float4 g1, float2 pa, float2 pb, float2 t,
                                            float2& sig, float2& alpha, float2& dx, float2& dy, float2& G,
                                            float2& a) {
    const float2 m1 = make_float2(-1.f, -1.f);
    dx = __ffma2_rn(__ffma2_rn(make_float2(g0.z, g0.z), t, make_float2(g0.x, g0.x)), m1, pa);
    dy = __ffma2_rn(__ffma2_rn(make_float2(g0.w, g0.w), t, make_float2(g0.y, g0.y)), m1, pb);
    if (LIDAR) dx = make_float2(wrap_pi(dx.x), wrap_pi(dx.y));
    const float ha = HALF ? g1.x : __fmul_rn(0.5f, g1.x), hc = HALF ? g1.z : __fmul_rn(0.5f, g1.z);
    const float2 u = __ffma2_rn(make_float2(ha, ha), dx, __fmul2_rn(make_float2(g1.y, g1.y), dy));
    sig = __ffma2_rn(dx, u, __fmul2_rn(__fmul2_rn(make_float2(hc, hc), dy), dy));
    const float2 e = __fmul2_rn(sig, make_float2(kNegLog2e, kNegLog2e));
    G = make_float2(exp2_approx(e.x), exp2_approx(e.y));
    a = __fmul2_rn(make_float2(g1.w, g1.w), G);   // before the 0.999 clamp
    alpha = make_float2(fminf(a.x, kAlphaMax), fminf(a.y, kAlphaMax));
}

struct FwdState {
    float T;
    int last;
    float de, dm;
    float los, cut;   // lidar line-of-sight term and its range cut r_p - eps
    bool med, done;
};

// Front-to-back blend of the tile's list for this thread's PX rays.  F may be null when
// only the transmittance and last index are wanted (recomputation).
template <int CM, int TW, int TH, bool LIDAR, int PX, bool WANT_F, bool COUNT = false>
__device__ __forceinline__ int forward_tile(Stage<CM, TW * TH / PX, LIDAR>& sm, const RasterIn& in,
                                            const TileCtx& tc, const TileBox& box, const RayCtx (&r)[PX],
                                            int2 range, FwdState (&st)[PX], float2 (*F)[CM / 2]) {
    constexpr int NT = TW * TH / PX, B = NT;   // one staged Gaussian per thread and batch
    int evals = 0;
    bool all_done = true;
#pragma unroll
    for (int q = 0; q < PX; q++) {
        st[q].T = 1.f;
        st[q].last = 0;
        st[q].de = 0.f;
        st[q].dm = 0.f;
        st[q].med = false;
        st[q].done = !r[q].inside;
        st[q].los = 0.f;
        st[q].cut = (LIDAR && in.los_range && r[q].inside) ? in.los_range[r[q].o] - in.los_eps : -INFINITY;
        all_done &= st[q].done;
    }
    float2 rpa[PX / 2 > 0 ? PX / 2 : 1], rpb[PX / 2 > 0 ? PX / 2 : 1], rt[PX / 2 > 0 ? PX / 2 : 1];   // ray pairs
#pragma unroll
    for (int qp = 0; qp < PX / 2; qp++) {
        rpa[qp] = make_float2(r[2 * qp].pa, r[2 * qp + 1].pa);
        rpb[qp] = make_float2(r[2 * qp].pb, r[2 * qp + 1].pb);
        rt[qp] = make_float2(r[2 * qp].t, r[2 * qp + 1].t);
    }
    // entries in groups of GU (each batch is padded with entries no ray blends); a thread
    // leaves after the group in which its rays finished.  Measured best: 4 (2, 8 and 16
    // are slower on the camera forward).
    constexpr int GU = 4;
    static_assert(B % GU == 0, "batches hold whole groups");
    __shared__ int s_wlive[NT / 32 > 0 ? NT / 32 : 1];
    for (int start = range.x; start < range.y; start += B) {
        if (__syncthreads_count(all_done) == NT) break;
        int nbg;   // staged entries of this batch, padded to whole groups
        if constexpr (!LIDAR) {
            // camera: only the entries that can reach alpha >= 1/255 somewhere in the tile are
            // staged, packed to the front in list order; live[] keeps each one's list position
            const int j = start + (int)threadIdx.x;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            uint32_t id = 0;
            float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
            bool lv = false;
            if (j < range.y) {
                id = load_id(in, j);
                g0 = in.rec[rec_index(tc.s, 0, in.n, id)];
                g1 = in.rec[rec_index(tc.s, 1, in.n, id)];
                lv = tile_live(g0, g1, box);
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, lv);
            if (lane == 0) s_wlive[warp] = __popc(bal);
            __syncthreads();
            int slot = __popc(bal & ((1u << lane) - 1u)), nlive = 0;
#pragma unroll
            for (int w = 0; w < NT / 32; w++) {
                const int c = s_wlive[w];
                slot += w < warp ? c : 0;
                nlive += c;
            }
            if (lv) {
                sm.g0[slot] = g0;
                sm.g1[slot] = make_float4(__fmul_rn(0.5f, g1.x), g1.y, __fmul_rn(0.5f, g1.z), g1.w);   // half conic
                sm.id[slot] = id;
                sm.live[slot] = j - range.x;
                const int C = in.C;
                const float* fp = in.feat + (int64_t)id * C;
                if ((C & 3) == 0) {
#pragma unroll
                    for (int c = 0; c < CM; c += 4)
                        if (c < C)
                            *reinterpret_cast<float4*>(&sm.f[slot * CM + c]) = *reinterpret_cast<const float4*>(fp + c);
                } else {
#pragma unroll
                    for (int c = 0; c < CM; c++)
                        if (c < C) sm.f[slot * CM + c] = fp[c];
                }
            }
            nbg = (nlive + GU - 1) / GU * GU;
            if ((int)threadIdx.x >= nlive && (int)threadIdx.x < nbg) {   // padding: no ray blends it
                sm.g0[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                sm.g1[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                sm.live[threadIdx.x] = 0;
#pragma unroll
                for (int c = 0; c < CM; c += 4)
                    *reinterpret_cast<float4*>(&sm.f[threadIdx.x * CM + c]) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
            if (start + (int)threadIdx.x < range.y) {
                stage_load<CM, B, LIDAR, true>(sm, in, tc.s, start + threadIdx.x, threadIdx.x, box);
            } else {   // past the list: an entry no ray blends (zero opacity, zero features)
                sm.g0[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                sm.g1[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                sm.g2[threadIdx.x] = make_float2(0.f, 0.f);
#pragma unroll
                for (int c = 0; c < CM; c += 4)
                    *reinterpret_cast<float4*>(&sm.f[threadIdx.x * CM + c]) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
            nbg = (min(B, range.y - start) + GU - 1) / GU * GU;
        }
        __syncthreads();
        if (!all_done) {
            for (int k0 = 0; k0 < nbg; k0 += GU) {
#pragma unroll
                for (int u = 0; u < GU; u++) {
                    const int k = k0 + u;
                    const float4 g0 = sm.g0[k], g1 = sm.g1[k];
                    all_done = true;
                    // alpha, the transmittance after the Gaussian and the blend weight of
                    // each ray; pairs of rays go through packed FP32 pairs
                    float av[PX], Tnv[PX], wv[PX];
                    bool ok[PX];
                    if constexpr (PX % 2 == 0) {
#pragma unroll
                        for (int qp = 0; qp < PX / 2; qp++) {
                            float2 sig2, a2, dx2, dy2, G2, au2;
                            eval_alpha2<LIDAR, true>(g0, g1, rpa[qp], rpb[qp], rt[qp], sig2, a2, dx2, dy2, G2, au2);
                            const float2 T2 = make_float2(st[2 * qp].T, st[2 * qp + 1].T);
                            const float2 w2 = __fmul2_rn(a2, T2);    // blend weight alpha T
                            // T (1 - alpha) as T - alpha T (one rounding, as __fsub_rn lane by lane)
                            const float2 Tn2 = __ffma2_rn(w2, make_float2(-1.f, -1.f), T2);
                            av[2 * qp] = a2.x;
                            av[2 * qp + 1] = a2.y;
                            Tnv[2 * qp] = Tn2.x;
                            Tnv[2 * qp + 1] = Tn2.y;
                            wv[2 * qp] = w2.x;
                            wv[2 * qp + 1] = w2.y;
                            ok[2 * qp] = sig2.x >= 0.f && a2.x >= kAlphaMin;
                            ok[2 * qp + 1] = sig2.y >= 0.f && a2.y >= kAlphaMin;
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < PX; q++) {
                            float dx, dy, G;
                            bool cl;
                            ok[q] = eval_alpha<LIDAR, true>(g0, g1, r[q], dx, dy, G, av[q], cl);
                            wv[q] = __fmul_rn(av[q], st[q].T);
                            Tnv[q] = __fsub_rn(st[q].T, wv[q]);
                        }
                    }
#pragma unroll
                    for (int q = 0; q < PX; q++) {
                        // Without branches: a ray that skips this Gaussian (finished, alpha
                        // below 1/255, or stopping before T would fall under 1e-4) takes
                        // weight 0, which leaves F, T and the ranges bit for bit unchanged.
                        if (COUNT) evals += st[q].done ? 0 : 1;
                        const float a = av[q], Tn = Tnv[q];
                        const bool hit = ok[q] && !st[q].done;
                        const bool stop = hit && Tn < kTEps;
                        const bool blend = hit && !stop;
                        st[q].done = st[q].done || stop;
                        const float wgt = blend ? wv[q] : 0.f;
                        if (WANT_F) {   // packed FP32 pairs: each lane is the same fused multiply-add
                            const float4* f4 = reinterpret_cast<const float4*>(sm.f + k * CM);
                            const float2 w2 = make_float2(wgt, wgt);
#pragma unroll
                            for (int c = 0; c < CM / 4; c++) {
                                const float4 v = f4[c];
                                F[q][2 * c] = __ffma2_rn(make_float2(v.x, v.y), w2, F[q][2 * c]);
                                F[q][2 * c + 1] = __ffma2_rn(make_float2(v.z, v.w), w2, F[q][2 * c + 1]);
                            }
                        }
                        if (LIDAR) {
                            const float rrs = sm.g2[k].x + sm.g2[k].y * r[q].t;
                            st[q].de += rrs * wgt;
                            if (blend && !st[q].med && Tn < 0.5f) {
                                st[q].dm = rrs;
                                st[q].med = true;
                            }
                            if (blend && rrs < st[q].cut) st[q].los += a;   // line-of-sight term (App. B)
                        }
                        st[q].T = blend ? Tn : st[q].T;
                        st[q].last = blend ? (LIDAR ? start + k - range.x : sm.live[k]) + 1 : st[q].last;
                        all_done = all_done && st[q].done;
                    }
                }
                if (all_done) break;
            }
        }
    }
    return evals;
}

// Resident blocks the camera forward asks the register allocator for: 20 warps per SM
// (24 spill).
template <int CM, bool LIDAR, int NT>
struct FwdMinBlocks {
    static constexpr int value = (!LIDAR && CM <= 16 && NT <= 640) ? 640 / NT : 1;
};

template <int CM, int TW, int TH, bool LIDAR, bool COUNT, bool LIST = false>
__global__ void __launch_bounds__(TW* TH / RaysPerThread<CM, false, LIDAR, TW * TH>::value,
                                  FwdMinBlocks<CM, LIDAR, TW * TH / RaysPerThread<CM, false, LIDAR, TW * TH>::value>::value)
    k_raster_fwd(const __grid_constant__ Frame fr, RasterIn in, RasterOut out) {
    constexpr int PX = RaysPerThread<CM, false, LIDAR, TW * TH>::value;
    constexpr int NT = TW * TH / PX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Stage<CM, NT, LIDAR>& sm = *reinterpret_cast<Stage<CM, NT, LIDAR>*>(smem_raw);
    TileCtx tc;
    RayCtx r[PX];
    if (!block_setup<TW, TH, LIDAR, LIST, PX, NT>(fr, in, tc, r)) return;
    const int2 range = load_range(in, tc.gtile);
    TileBox box{};
    if (!LIDAR) box = camera_tile_box(fr.s[tc.s], tc.tx, tc.ty, TW, TH);
    float2 F[PX][CM / 2];
#pragma unroll
    for (int q = 0; q < PX; q++)
#pragma unroll
        for (int c = 0; c < CM / 2; c++) F[q][c] = make_float2(0.f, 0.f);
    FwdState st[PX];
    const int evals = forward_tile<CM, TW, TH, LIDAR, PX, true, COUNT>(sm, in, tc, box, r, range, st, F);
    if (COUNT) {
        unsigned long long e = (unsigned long long)evals;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(out.evaluated, e);
    }
    const int C = in.C;
    if (!LIDAR && out.l1_grad) {
        // fused L1 term (Eq. loss_fn): the gradient image and one loss atomic per block
        float acc = 0.f;
        const float sc = out.l1_scale;
        auto sg = [sc](float d) { return d > 0.f ? sc : (d < 0.f ? -sc : 0.f); };
#pragma unroll
        for (int q = 0; q < PX; q++) {
            if (!r[q].inside) continue;
            const float* tg = out.l1_target + r[q].o * C;
            float* gd = out.l1_grad + r[q].o * C;
            if ((C & 3) == 0) {
#pragma unroll
                for (int c = 0; c < CM; c += 4) {
                    if (c < C) {
                        const float4 t = *reinterpret_cast<const float4*>(tg + c);
                        const float d0 = F[q][c / 2].x - t.x, d1 = F[q][c / 2].y - t.y;
                        const float d2 = F[q][c / 2 + 1].x - t.z, d3 = F[q][c / 2 + 1].y - t.w;
                        acc += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
                        *reinterpret_cast<float4*>(gd + c) = make_float4(sg(d0), sg(d1), sg(d2), sg(d3));
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < CM; c++) {
                    if (c < C) {
                        const float d = ((c & 1) ? F[q][c / 2].y : F[q][c / 2].x) - tg[c];
                        acc += fabsf(d);
                        gd[c] = sg(d);
                    }
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        __shared__ float s_l1[NT / 32 > 0 ? NT / 32 : 1];
        if ((threadIdx.x & 31) == 0) s_l1[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            float tot = 0.f;
            for (int w = 0; w < NT / 32; w++) tot += s_l1[w];
            if (tot != 0.f) atomicAdd(out.l1_loss, tot * sc);
        }
    }
#pragma unroll
    for (int q = 0; q < PX; q++) {
        if (!r[q].inside) continue;
        if (!out.feat) continue;
        float* fo = out.feat + r[q].o * C;
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
        if (out.T) out.T[r[q].o] = st[q].T;
        if (out.last) out.last[r[q].o] = st[q].last;
        if (LIDAR) {
            out.range_exp[r[q].o] = st[q].de;
            if (out.los) out.los[r[q].o] = st[q].los;
            if (out.range_med) out.range_med[r[q].o] = st[q].dm;
            out.alpha[r[q].o] = 1.f - st[q].T;
        }
    }
}

// Sum of VP per-lane values over the warp.  At each of the five butterfly steps
// (lane offsets 16, 8, 4, 2, 1) an even count n is halved: a lane keeps one half of its
// values and receives the partner's copy of that half; an odd count is summed whole.
// Afterwards lane l holds the totals of the value indices
// [reduce_first<VP>(l), reduce_first<VP>(l) + reduce_left<VP>()); the lanes of a replica
// group share them out for reporting, one value per lane per round.
__host__ __device__ constexpr int reduce_left_n(int n, int step) {
    return step == 5 ? n : reduce_left_n((n >= 2 && n % 2 == 0) ? n / 2 : n, step + 1);
}
template <int VP>
__host__ __device__ constexpr int reduce_left() { return reduce_left_n(VP, 0); }

// Issue cost of the reduction (shuffles, selects and adds) for a padded count VP.
__host__ __device__ constexpr int reduce_cost(int n, int step = 0) {
    return step == 5 ? 0
                     : ((n >= 2 && n % 2 == 0) ? 2 * n + reduce_cost(n / 2, step + 1)
                                               : 2 * n + reduce_cost(n, step + 1));
}
// Cheapest padded count >= v (halving steps move half the values at 4 instructions each;
// whole sums move every value at 2).
__host__ __device__ constexpr int reduce_pad(int v, int best = 0, int p = 0) {
    return p == 0 ? reduce_pad(v, v, v + 1)
                  : (p > 64 ? best : reduce_pad(v, reduce_cost(p) < reduce_cost(best) ? p : best, p + 1));
}

// Number of trailing whole-sum steps: lanes that differ only in those low bits hold the
// same totals afterwards (a replica group of 1 << reduce_plain() lanes).
__host__ __device__ constexpr int reduce_plain_n(int n, int step) {
    return step == 5 ? 0
                     : ((n >= 2 && n % 2 == 0) ? reduce_plain_n(n / 2, step + 1) : 1 + reduce_plain_n(n, step + 1));
}
template <int VP>
__host__ __device__ constexpr int reduce_plain() { return reduce_plain_n(VP, 0); }

template <int VP>
__device__ __forceinline__ int reduce_first(int lane) {
    int n = VP, j0 = 0;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        if (n >= 2 && n % 2 == 0) {
            n /= 2;
            if (lane & o) j0 += n;
        }
    }
    return j0;
}

template <int VP>
__device__ __forceinline__ void warp_transpose_reduce(float (&v)[VP], int lane) {
    int n = VP;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
        if (n >= 2 && n % 2 == 0) {
            const int h = n / 2;
            float recv[VP / 2];
#pragma unroll
            for (int i = 0; i < VP / 2; i++) {
                if (i < h) {
                    const float send = upper ? v[i] : v[i + h];
                    v[i] = upper ? v[i + h] : v[i];
                    recv[i] = __shfl_xor_sync(0xffffffffu, send, o);
                }
            }
            // the adds two at a time (packed FP32 pairs; the same IEEE additions)
#pragma unroll
            for (int i = 0; i + 1 < VP / 2; i += 2) {
                if (i + 1 < h) {
                    const float2 s2 = __fadd2_rn(make_float2(v[i], v[i + 1]), make_float2(recv[i], recv[i + 1]));
                    v[i] = s2.x;
                    v[i + 1] = s2.y;
                } else if (i < h) {
                    v[i] += recv[i];
                }
            }
            n = h;
        } else {
            float recv[VP];
#pragma unroll
            for (int i = 0; i < VP; i++)
                if (i < n) recv[i] = __shfl_xor_sync(0xffffffffu, v[i], o);
#pragma unroll
            for (int i = 0; i + 1 < VP; i += 2) {
                if (i + 1 < n) {
                    const float2 s2 = __fadd2_rn(make_float2(v[i], v[i + 1]), make_float2(recv[i], recv[i + 1]));
                    v[i] = s2.x;
                    v[i + 1] = s2.y;
                } else if (i < n) {
                    v[i] += recv[i];
                }
            }
        }
    }
}

// One halving butterfly step on v[0, 2H): the lane with lane bit `o` set keeps the high
// half, the other the low half; each receives the partner's copy of the half it keeps.
template <int H, int VP>
__device__ __forceinline__ void halve_step(float (&v)[VP], int lane, int o) {
    const bool up = (lane & o) != 0;
    float sd[H], kp[H];
#pragma unroll
    for (int i = 0; i < H; i++) {
        sd[i] = up ? v[i] : v[i + H];
        kp[i] = up ? v[i + H] : v[i];
    }
#pragma unroll
    for (int i = 0; i < H; i++) sd[i] = __shfl_xor_sync(0xffffffffu, sd[i], o);
#pragma unroll
    for (int i = 0; i < H; i += 2) {
        if (i + 1 < H) {
            const float2 s2 = __fadd2_rn(make_float2(kp[i], kp[i + 1]), make_float2(sd[i], sd[i + 1]));
            v[i] = s2.x;
            v[i + 1] = s2.y;
        } else {
            v[i] = kp[i] + sd[i];
        }
    }
}

template <int NSL>
__device__ __forceinline__ void acc_put(float* row, int j, float val) {
    if (NSL > 1) row[j] = val;                       // this warp's own slice
    else if (val != 0.f) atomicAdd(&row[j], val);    // one slice shared by the warps
}

// Camera backward: the warp sums of an entry's 8 geometric values v[0, 8) and its CM
// feature values v[8, 8 + CM), the features in the lane's chunk order (register chunk c =
// channel chunk c ^ m2).  The features' chunk steps need no selects: at lane bit 4 (and 3
// for 16 channels) each lane keeps its low chunks and sends its high ones.  Two halving
// steps then split the last chunk, whole sums finish the remaining lane bits.  The
// geometric values take three halving steps (lane bits 4, 3, 2) and two whole sums.  Each
// total is reported once: geometric value (lane >> 2) & 7 by the lanes with low bits 00,
// the feature channel of the lane by the lanes with no whole-sum bit set.
template <int CM, int VP, int NSL>
__device__ __forceinline__ void reduce_report_camera(float (&v)[VP], int lane, float* row, int nfeat) {
    constexpr int OFF = 8;
    constexpr int SC = CM >= 16 ? 2 : (CM >= 8 ? 1 : 0);
    constexpr int O1 = 16 >> SC, O2 = O1 >> 1;   // lane bits of the two in-chunk steps
    static_assert(OFF + CM <= VP, "camera values");
#pragma unroll
    for (int st = 0; st < SC; st++) {
        const int o = 16 >> st, h = CM >> (st + 1);
        float rc[CM / 2];
#pragma unroll
        for (int p = 0; p < CM / 2; p++)
            if (p < h) rc[p] = __shfl_xor_sync(0xffffffffu, v[OFF + p + h], o);
#pragma unroll
        for (int p = 0; p < CM / 2; p += 2) {
            if (p < h) {
                const float2 s2 = __fadd2_rn(make_float2(v[OFF + p], v[OFF + p + 1]), make_float2(rc[p], rc[p + 1]));
                v[OFF + p] = s2.x;
                v[OFF + p + 1] = s2.y;
            }
        }
    }
    {   // the chunk's four values: keep a pair, then one of it
        float c4[4] = {v[OFF], v[OFF + 1], v[OFF + 2], v[OFF + 3]};
        halve_step<2>(c4, lane, O1);
        halve_step<1>(c4, lane, O2);
        float f = c4[0];
#pragma unroll
        for (int o = O2 >> 1; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        v[OFF] = f;
    }
    halve_step<4>(v, lane, 16);
    halve_step<2>(v, lane, 8);
    halve_step<1>(v, lane, 4);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    const int m2 = (lane >> (5 - SC)) & ((1 << SC) - 1);
    const int ch = 4 * m2 + ((lane & O1) ? 2 : 0) + ((lane & O2) ? 1 : 0);
    if ((lane & 3) == 0) acc_put<NSL>(row, (lane >> 2) & 7, v[0]);
    if ((lane & (O2 - 1)) == 0 && ch < nfeat) acc_put<NSL>(row, OFF + ch, v[OFF]);
}

// Resident blocks the camera backward asks the register allocator for: 12 warps per SM
// (unbounded, the packed loops take registers enough to drop to 10; 14 would spill).
template <int CM, bool LIDAR, int NT>
struct BwdMinBlocks {
    static constexpr int value = (!LIDAR && CM <= 16 && NT <= 384) ? 384 / NT : 1;
};

template <int CM, bool LIDAR>
struct BwdLayout {
    static constexpr int kOffF = LIDAR ? 12 : 8;          // first feature slot (16-byte aligned)
    static constexpr int kV = kOffF + CM;                 // values per (ray, Gaussian)
    static constexpr int kVP = reduce_pad(kV);            // padded count for the warp reduction
    static constexpr int kRow = (kV + 3) & ~3;            // shared accumulator row (float4 aligned)
    // With at most two warps per tile each warp keeps its own accumulator slice and stores
    // its per-Gaussian totals without atomics; the flush adds the slices.
    __host__ __device__ static constexpr int slices(int warps) { return warps <= 2 ? warps : 1; }
};

template <int CM, int TW, int TH, bool LIDAR, bool RECOMPUTE, bool LIST = false>
__global__ void __launch_bounds__(TW* TH / RaysPerThread<CM, true, LIDAR, TW * TH>::value,
                                  BwdMinBlocks<CM, LIDAR, TW * TH / RaysPerThread<CM, true, LIDAR, TW * TH>::value>::value)
    k_raster_bwd(const __grid_constant__ Frame fr, RasterIn in, RasterGrad gr) {
    constexpr int PX = RaysPerThread<CM, true, LIDAR, TW * TH>::value;
    constexpr int NT = TW * TH / PX;
    constexpr int B = NT;   // one staged Gaussian per thread and batch
    using LY = BwdLayout<CM, LIDAR>;
    constexpr int OFF = LY::kOffF, VP = LY::kVP, ROW = LY::kRow;
    constexpr int NSL = LY::slices(NT / 32);   // accumulator slices (1: shared by all warps, atomics)
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Stage<CM, B, LIDAR>& sm = *reinterpret_cast<Stage<CM, B, LIDAR>*>(smem_raw);
    float* acc = reinterpret_cast<float*>(smem_raw + sizeof(Stage<CM, B, LIDAR>));   // [NSL][B][ROW]
    __shared__ int s_max_last[NT / 32 > 0 ? NT / 32 : 1];
    const int Crt = in.C;
    const int V = OFF + Crt;
    TileCtx tc;
    RayCtx r[PX];
    if (!block_setup<TW, TH, LIDAR, LIST, PX, NT>(fr, in, tc, r)) return;
    float2 rpa[PX / 2 > 0 ? PX / 2 : 1], rpb[PX / 2 > 0 ? PX / 2 : 1], rt[PX / 2 > 0 ? PX / 2 : 1];   // ray pairs
#pragma unroll
    for (int qp = 0; qp < PX / 2; qp++) {
        rpa[qp] = make_float2(r[2 * qp].pa, r[2 * qp + 1].pa);
        rpb[qp] = make_float2(r[2 * qp].pb, r[2 * qp + 1].pb);
        rt[qp] = make_float2(r[2 * qp].t, r[2 * qp + 1].t);
    }
    const int2 range = load_range(in, tc.gtile);
    const int len = range.y - range.x;
    TileBox box{};
    if (!LIDAR) box = camera_tile_box(fr.s[tc.s], tc.tx, tc.ty, TW, TH);
    for (int q = threadIdx.x; q < NSL * B * ROW; q += NT) acc[q] = 0.f;
    float Tfin[PX];
    int last[PX];
    if (RECOMPUTE) {
        FwdState st[PX];
        forward_tile<CM, TW, TH, LIDAR, PX, false>(sm, in, tc, box, r, range, st, nullptr);
#pragma unroll
        for (int q = 0; q < PX; q++) {
            Tfin[q] = st[q].T;
            last[q] = min(st[q].last, len);
        }
    } else {
#pragma unroll
        for (int q = 0; q < PX; q++) {
            Tfin[q] = r[q].inside ? gr.T[r[q].o] : 1.f;
            last[q] = r[q].inside ? min(gr.last[r[q].o], len) : 0;   // never past this tile's list
        }
    }
    float2 gF[PX][CM / 2];   // upstream feature gradient, as FP32 pairs for the packed FMAs
    // Camera (rays in pairs): the feature sums of an entry are reduced over the warp with
    // select-free butterfly steps.  Lane l holds its channels in a lane-dependent chunk
    // order -- register chunk c is channel chunk c ^ m2, m2 = the lane bits of the chunk
    // steps -- and reads each Gaussian's features in the same order, so at each chunk step
    // every lane keeps its low registers and sends its high ones, the partner's high
    // registers being the channels of its own low ones.
    constexpr bool kSplitRed = !LIDAR && PX % 2 == 0;
    constexpr int kChunkSteps = CM >= 16 ? 2 : (CM >= 8 ? 1 : 0);
    static_assert(!kSplitRed || (CM >= 4 && CM <= 16 && (CM & (CM - 1)) == 0), "chunked feature reduction");
    const int m2 = kSplitRed ? (((int)threadIdx.x & 31) >> (5 - kChunkSteps)) & ((1 << kChunkSteps) - 1) : 0;
    float gTT[PX], gD[PX], T[PX], S[PX], SD[PX];
    float gL[PX], cut[PX];   // lidar line-of-sight upstream gradient and range cut
    float dtime = 0.f;       // camera: this thread's share of dL/d (camera time offset)
    int my_last = 0;
#pragma unroll
    for (int q = 0; q < PX; q++) {
#pragma unroll
        for (int c = 0; c < CM / 2; c++) {
            const int c0 = kSplitRed ? 4 * ((c >> 1) ^ m2) + 2 * (c & 1) : 2 * c, c1 = c0 + 1;
            gF[q][c] = make_float2((r[q].inside && c0 < Crt) ? gr.dfeat[r[q].o * Crt + c0] : 0.f,
                                   (r[q].inside && c1 < Crt) ? gr.dfeat[r[q].o * Crt + c1] : 0.f);
        }
        float gT = 0.f;
        gD[q] = 0.f;
        if (r[q].inside) {
            if (!LIDAR) {
                gT = gr.dT ? gr.dT[r[q].o] : 0.f;
            } else {
                gT = gr.dalpha ? -gr.dalpha[r[q].o] : 0.f;
                gD[q] = gr.drange ? gr.drange[r[q].o] : 0.f;
            }
        }
        gTT[q] = gT * Tfin[q];
        gL[q] = (LIDAR && gr.dlos && r[q].inside) ? gr.dlos[r[q].o] : 0.f;
        cut[q] = (LIDAR && in.los_range && r[q].inside) ? in.los_range[r[q].o] - in.los_eps : -INFINITY;
        T[q] = Tfin[q];
        S[q] = 0.f;    // sum_c gF_c B_c, B = normalised blend of everything behind
        SD[q] = 0.f;   // its counterpart for the range
        my_last = max(my_last, last[q]);
    }
    const int wl = __reduce_max_sync(0xffffffffu, (unsigned)my_last);   // this warp's deepest entry
    if ((threadIdx.x & 31) == 0) s_max_last[threadIdx.x >> 5] = wl;
    __syncthreads();
    int max_last = 0;
#pragma unroll
    for (int w = 0; w < (NT + 31) / 32; w++) max_last = max(max_last, s_max_last[w]);
    const int lane = threadIdx.x & 31;
    float4* gp0 = gr.grad_proj + rec_index(tc.s, 0, in.n, 0);
    float4* gp1 = gr.grad_proj + rec_index(tc.s, 1, in.n, 0);
    float4* gp2 = gr.grad_proj + rec_index(tc.s, 2, in.n, 0);
    for (int end = range.x + max_last; end > range.x; end -= B) {
        const int cnt = min(B, end - range.x);
        __syncthreads();
        if ((int)threadIdx.x < cnt) stage_load<CM, B, LIDAR>(sm, in, tc.s, end - 1 - threadIdx.x, threadIdx.x, box);
        __syncthreads();
        for (int k = 0; k < cnt; k++) {
            const int idx = end - 1 - k - range.x;
            if (idx >= wl) continue;   // warp-uniform: no ray of this warp blended this deep
            if (!LIDAR && !sm.live[k]) continue;   // no pixel of the tile can blend it
            const float4 g0 = sm.g0[k], g1 = sm.g1[k];
            float v[VP];
            if constexpr (PX % 2 == 0) {
                // pairs of rays in packed FP32 pairs: the same per-ray chain as below, two
                // lanes at a time; the eight geometric terms are accumulated over the pairs
                constexpr int NP = PX / 2;
                float2 dx2[NP], dy2[NP], G2[NP], a2[NP];
                bool on[PX], cl[PX];
                bool any = false;
#pragma unroll
                for (int qp = 0; qp < NP; qp++) {
                    float2 sig2, au2;
                    eval_alpha2<LIDAR>(g0, g1, rpa[qp], rpb[qp], rt[qp], sig2, a2[qp], dx2[qp], dy2[qp], G2[qp], au2);
                    on[2 * qp] = sig2.x >= 0.f && a2[qp].x >= kAlphaMin && idx < last[2 * qp];
                    on[2 * qp + 1] = sig2.y >= 0.f && a2[qp].y >= kAlphaMin && idx < last[2 * qp + 1];
                    cl[2 * qp] = au2.x > kAlphaMax;
                    cl[2 * qp + 1] = au2.y > kAlphaMax;
                    any |= on[2 * qp] || on[2 * qp + 1];
                }
                if (!__any_sync(0xffffffffu, any)) continue;
                const float2 m1 = make_float2(-1.f, -1.f);
                float2 acc[LIDAR ? 10 : 8];
                float2 vf[CM / 2];   // feature-gradient terms, accumulated as packed pairs
#pragma unroll
                for (int qp = 0; qp < NP; qp++) {
                    const int q0 = 2 * qp, q1 = 2 * qp + 1;
                    // a ray that does not blend this Gaussian gets alpha = 0: every term vanishes
                    const float2 aq = make_float2(on[q0] ? a2[qp].x : 0.f, on[q1] ? a2[qp].y : 0.f);
                    const float2 Gq = make_float2(on[q0] ? G2[qp].x : 0.f, on[q1] ? G2[qp].y : 0.f);
                    const float2 om = __ffma2_rn(aq, m1, make_float2(1.f, 1.f));
                    const float2 inv = make_float2(rcp_approx(om.x), rcp_approx(om.y));
                    const float2 Ti = __fmul2_rn(make_float2(T[q0], T[q1]), inv);
                    const float2 wgt = __fmul2_rn(aq, Ti);
                    float Gf[2];
#pragma unroll
                    for (int j = 0; j < 2; j++) {   // sum_c gF_c f_c, two interleaved partial sums
                        const float4* f4 = reinterpret_cast<const float4*>(sm.f + k * CM);
                        float2 g2 = make_float2(0.f, 0.f);
#pragma unroll
                        for (int c = 0; c < CM / 4; c++) {
                            const float4 fv = f4[c ^ m2];   // the lane's chunk order
                            g2 = __ffma2_rn(gF[q0 + j][2 * c], make_float2(fv.x, fv.y), g2);
                            g2 = __ffma2_rn(gF[q0 + j][2 * c + 1], make_float2(fv.z, fv.w), g2);
                        }
                        Gf[j] = g2.x + g2.y;
                    }
                    const float2 S2 = make_float2(S[q0], S[q1]);
                    const float2 dS = __ffma2_rn(S2, m1, make_float2(Gf[0], Gf[1]));   // Gf - S
                    float2 dal = __ffma2_rn(Ti, dS, __fmul2_rn(make_float2(-gTT[q0], -gTT[q1]), inv));
                    const float2 Sn = __ffma2_rn(aq, dS, S2);
                    S[q0] = Sn.x;
                    S[q1] = Sn.y;
                    float2 drrs = make_float2(0.f, 0.f);
                    if (LIDAR) {
                        const float2 rrs = __ffma2_rn(make_float2(sm.g2[k].y, sm.g2[k].y), rt[qp],
                                                      make_float2(sm.g2[k].x, sm.g2[k].x));
                        const float2 SD2 = make_float2(SD[q0], SD[q1]);
                        const float2 eD = __ffma2_rn(SD2, m1, rrs);   // r_rs - SD
                        const float2 gD2 = make_float2(gD[q0], gD[q1]);
                        dal = __ffma2_rn(__fmul2_rn(Ti, gD2), eD, dal);
                        if (rrs.x < cut[q0]) dal.x += gL[q0];   // d(line-of-sight term) / d alpha
                        if (rrs.y < cut[q1]) dal.y += gL[q1];
                        const float2 SDn = __ffma2_rn(aq, eD, SD2);
                        SD[q0] = SDn.x;
                        SD[q1] = SDn.y;
                        drrs = __fmul2_rn(gD2, wgt);
                    }
                    // clamped alpha (o' G > 0.999) passes no gradient to o' and the exponent
                    const float2 dg = make_float2((on[q0] && !cl[q0]) ? dal.x : 0.f, (on[q1] && !cl[q1]) ? dal.y : 0.f);
                    const float2 P = __fmul2_rn(dg, aq);   // -dL/dsigma
                    const float2 Kx = __ffma2_rn(make_float2(g1.x, g1.x), dx2[qp],
                                                 __fmul2_rn(make_float2(g1.y, g1.y), dy2[qp]));
                    const float2 Ky = __ffma2_rn(make_float2(g1.y, g1.y), dx2[qp],
                                                 __fmul2_rn(make_float2(g1.z, g1.z), dy2[qp]));
                    const float2 nddx = __fmul2_rn(P, Kx), nddy = __fmul2_rn(P, Ky);   // -ddx, -ddy
                    const float2 hx = __fmul2_rn(P, dx2[qp]), hy = __fmul2_rn(P, dy2[qp]);
                    const float2 tq = rt[qp];
                    if (qp == 0) {
                        acc[0] = nddx;
                        acc[1] = nddy;
                        acc[2] = __fmul2_rn(nddx, tq);
                        acc[3] = __fmul2_rn(nddy, tq);
                        acc[4] = __fmul2_rn(hx, dx2[qp]);
                        acc[5] = __fmul2_rn(hx, dy2[qp]);
                        acc[6] = __fmul2_rn(hy, dy2[qp]);
                        acc[7] = __fmul2_rn(dg, Gq);
                        if constexpr (LIDAR) {
                            acc[8] = drrs;
                            acc[9] = __fmul2_rn(drrs, tq);
                        }
#pragma unroll
                        for (int c = 0; c < CM / 2; c++) vf[c] = __fmul2_rn(make_float2(wgt.x, wgt.x), gF[q0][c]);
                    } else {
                        acc[0] = __fadd2_rn(acc[0], nddx);
                        acc[1] = __fadd2_rn(acc[1], nddy);
                        acc[2] = __ffma2_rn(nddx, tq, acc[2]);
                        acc[3] = __ffma2_rn(nddy, tq, acc[3]);
                        acc[4] = __ffma2_rn(hx, dx2[qp], acc[4]);
                        acc[5] = __ffma2_rn(hx, dy2[qp], acc[5]);
                        acc[6] = __ffma2_rn(hy, dy2[qp], acc[6]);
                        acc[7] = __ffma2_rn(dg, Gq, acc[7]);
                        if constexpr (LIDAR) {
                            acc[8] = __fadd2_rn(acc[8], drrs);
                            acc[9] = __ffma2_rn(drrs, tq, acc[9]);
                        }
#pragma unroll
                        for (int c = 0; c < CM / 2; c++)
                            vf[c] = __ffma2_rn(make_float2(wgt.x, wgt.x), gF[q0][c], vf[c]);
                    }
#pragma unroll
                    for (int c = 0; c < CM / 2; c++) vf[c] = __ffma2_rn(make_float2(wgt.y, wgt.y), gF[q1][c], vf[c]);
                    T[q0] = Ti.x;
                    T[q1] = Ti.y;
                }
                // (-ddx, -ddy, -ddx t, -ddy t, dsig dx^2 / 2, dsig dx dy, dsig dy^2 / 2, dg G) summed
                // over this thread's rays; dsig = -P
                v[0] = acc[0].x + acc[0].y;
                v[1] = acc[1].x + acc[1].y;
                v[2] = acc[2].x + acc[2].y;
                v[3] = acc[3].x + acc[3].y;
                v[4] = -0.5f * (acc[4].x + acc[4].y);
                v[5] = -(acc[5].x + acc[5].y);
                v[6] = -0.5f * (acc[6].x + acc[6].y);
                v[7] = acc[7].x + acc[7].y;
#pragma unroll
                for (int j = 8; j < OFF; j++) v[j] = 0.f;
                if constexpr (LIDAR) {
                    v[8] = acc[8].x + acc[8].y;
                    v[9] = acc[9].x + acc[9].y;
                }
                // every pixel time carries the camera time offset; the mean moves by v t
                if (!LIDAR && gr.dsensor) dtime += v[0] * g0.z + v[1] * g0.w;
#pragma unroll
                for (int c = 0; c < CM / 2; c++) {
                    v[OFF + 2 * c] = vf[c].x;
                    v[OFF + 2 * c + 1] = vf[c].y;
                }
#pragma unroll
                for (int j = OFF + CM; j < VP; j++) v[j] = 0.f;
            } else {
                float dx[PX], dy[PX], G[PX], a[PX];
                bool cl[PX], on[PX];
                bool any = false;
#pragma unroll
                for (int q = 0; q < PX; q++) {
                    on[q] = eval_alpha<LIDAR>(g0, g1, r[q], dx[q], dy[q], G[q], a[q], cl[q]) && idx < last[q];
                    any |= on[q];
                }
                if (!__any_sync(0xffffffffu, any)) continue;
                float2 vf[CM / 2];   // feature-gradient terms, accumulated as packed pairs
#pragma unroll
                for (int q = 0; q < PX; q++) {
                    // a ray that does not blend this Gaussian gets alpha = 0: every term vanishes
                    const float aq = on[q] ? a[q] : 0.f;
                    const float Gq = on[q] ? G[q] : 0.f;
                    const float inv = rcp_approx(1.f - aq);   // 1 - alpha >= 0.001: no special cases
                    const float Ti = T[q] * inv;
                    const float wgt = aq * Ti;
                    // sum_c gF_c f_c in two interleaved partial sums (packed FP32 pairs)
                    const float4* f4 = reinterpret_cast<const float4*>(sm.f + k * CM);
                    float2 g2 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int c = 0; c < CM / 4; c++) {
                        const float4 fv = f4[c];
                        g2 = __ffma2_rn(gF[q][2 * c], make_float2(fv.x, fv.y), g2);
                        g2 = __ffma2_rn(gF[q][2 * c + 1], make_float2(fv.z, fv.w), g2);
                    }
                    const float Gf = g2.x + g2.y;
                    float dalpha = Ti * (Gf - S[q]) - gTT[q] * inv;
                    S[q] += aq * (Gf - S[q]);
                    float drrs = 0.f, tq = r[q].t;
                    if (LIDAR) {
                        const float rrs = sm.g2[k].x + sm.g2[k].y * tq;
                        dalpha += Ti * gD[q] * (rrs - SD[q]);
                        if (rrs < cut[q]) dalpha += gL[q];   // d(line-of-sight term) / d alpha
                        SD[q] += aq * (rrs - SD[q]);
                        drrs = gD[q] * wgt;
                    }
                    // clamped alpha (o' G > 0.999) passes no gradient to o' and the exponent
                    const float dg = (on[q] && !cl[q]) ? dalpha : 0.f;
                    const float dsig = -dg * aq;
                    const float ddx = dsig * (g1.x * dx[q] + g1.y * dy[q]);
                    const float ddy = dsig * (g1.y * dx[q] + g1.z * dy[q]);
                    const float t0[8] = {-ddx, -ddy, -ddx * tq, -ddy * tq, dsig * 0.5f * dx[q] * dx[q],
                                         dsig * dx[q] * dy[q], dsig * 0.5f * dy[q] * dy[q], dg * Gq};
                    // every pixel time carries the camera time offset; the mean moves by v t
                    if (!LIDAR && gr.dsensor) dtime += t0[0] * g0.z + t0[1] * g0.w;
                    if (q == 0) {
#pragma unroll
                        for (int j = 0; j < 8; j++) v[j] = t0[j];
#pragma unroll
                        for (int j = 8; j < OFF; j++) v[j] = 0.f;
#pragma unroll
                        for (int c = 0; c < CM / 2; c++) vf[c] = __fmul2_rn(make_float2(wgt, wgt), gF[q][c]);
#pragma unroll
                        for (int j = OFF + CM; j < VP; j++) v[j] = 0.f;
                        if (LIDAR) {
                            v[8] = drrs;
                            v[9] = drrs * tq;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 8; j++) v[j] += t0[j];
#pragma unroll
                        for (int c = 0; c < CM / 2; c++) vf[c] = __ffma2_rn(make_float2(wgt, wgt), gF[q][c], vf[c]);
                        if (LIDAR) {
                            v[8] += drrs;
                            v[9] += drrs * tq;
                        }
                    }
                    T[q] = Ti;
                }
#pragma unroll
                for (int c = 0; c < CM / 2; c++) {
                    v[OFF + 2 * c] = vf[c].x;
                    v[OFF + 2 * c + 1] = vf[c].y;
                }
            }
            if constexpr (kSplitRed) {
                reduce_report_camera<CM, VP, NSL>(v, lane, acc + ((NSL > 1 ? (threadIdx.x >> 5) * B : 0) + k) * ROW,
                                                  Crt);
                continue;
            }
            warp_transpose_reduce<VP>(v, lane);
            constexpr int M = reduce_left<VP>(), RG = 1 << reduce_plain<VP>();
            const int j0 = reduce_first<VP>(lane), rank = lane & (RG - 1);
#pragma unroll
            for (int q0 = 0; q0 < M; q0 += RG) {
                float val = v[q0];
#pragma unroll
                for (int q = q0 + 1; q < q0 + RG && q < M; q++) val = (rank == q - q0) ? v[q] : val;
                const int j = j0 + q0 + rank;
                if (NSL > 1) {
                    if (q0 + rank < M && j < V) acc[((threadIdx.x >> 5) * B + k) * ROW + j] = val;
                } else if (q0 + rank < M && j < V && val != 0.f) {
                    atomicAdd(&acc[k * ROW + j], val);
                }
            }
        }
        __syncthreads();
        // one set of vector atomics per (tile, Gaussian): flush this batch's sums
        if ((int)threadIdx.x < cnt) {
            const int slot = threadIdx.x;
            float* a_row = acc + slot * ROW;
#pragma unroll
            for (int w = 1; w < NSL; w++) {   // fold the other warps' slices into the first
                float* o_row = acc + (w * B + slot) * ROW;
#pragma unroll
                for (int q = 0; q < ROW; q += 4) {
                    float4 x = *reinterpret_cast<float4*>(a_row + q);
                    const float4 y = *reinterpret_cast<float4*>(o_row + q);
                    x.x += y.x;
                    x.y += y.y;
                    x.z += y.z;
                    x.w += y.w;
                    *reinterpret_cast<float4*>(a_row + q) = x;
                    *reinterpret_cast<float4*>(o_row + q) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            const uint32_t id = sm.id[slot];
            const float4 s0 = *reinterpret_cast<float4*>(a_row);
            const float4 s1 = *reinterpret_cast<float4*>(a_row + 4);
            if (s0.x != 0.f || s0.y != 0.f || s0.z != 0.f || s0.w != 0.f || s1.x != 0.f || s1.y != 0.f ||
                s1.z != 0.f || s1.w != 0.f) {
                atomicAdd(gp0 + id, s0);
                atomicAdd(gp1 + id, s1);
            }
            if (LIDAR) {
                const float2 s2 = make_float2(a_row[8], a_row[9]);
                if (s2.x != 0.f || s2.y != 0.f) atomicAdd(reinterpret_cast<float2*>(gp2 + id), s2);
            }
            float* df = gr.dfeatures + (int64_t)id * Crt;
            if ((Crt & 3) == 0) {
#pragma unroll
                for (int c = 0; c < CM; c += 4) {
                    if (c < Crt) {
                        const float4 f4 = *reinterpret_cast<float4*>(a_row + OFF + c);
                        if (f4.x != 0.f || f4.y != 0.f || f4.z != 0.f || f4.w != 0.f)
                            atomicAdd(reinterpret_cast<float4*>(df + c), f4);
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < CM; c++)
                    if (c < Crt && a_row[OFF + c] != 0.f) atomicAdd(df + c, a_row[OFF + c]);
            }
#pragma unroll
            for (int q = 0; q < ROW; q += 4) *reinterpret_cast<float4*>(a_row + q) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    if (!LIDAR && gr.dsensor) {   // one atomic per block (uniform branch)
        __shared__ float s_dt[NT / 32 > 0 ? NT / 32 : 1];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dtime += __shfl_xor_sync(0xffffffffu, dtime, o);
        if (lane == 0) s_dt[threadIdx.x >> 5] = dtime;
        __syncthreads();
        if (threadIdx.x == 0) {
            float tot = 0.f;
            for (int w = 0; w < NT / 32; w++) tot += s_dt[w];
            if (tot != 0.f) atomicAdd(gr.dsensor + 16 * tc.s + 6, tot);
        }
    }
}

}  // namespace splat

#include "raster_bwd_mma.cuh"   // the 16-channel camera backward on the tensor cores

namespace splat {

// ---------------------------------------------------------------------------------
// Host launch helpers (instantiated per channel bucket in raster_c*.cu)
// ---------------------------------------------------------------------------------

template <typename K>
static void set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int CM, int TW, int TH, bool LIDAR>
static void launch_fwd_t(const Frame& fr, int blocks, const RasterIn& in, const RasterOut& out, cudaStream_t st) {
    constexpr int NT = TW * TH / RaysPerThread<CM, false, LIDAR, TW * TH>::value;
    const size_t sm = sizeof(Stage<CM, NT, LIDAR>);
    // the evaluated-pair counter is compiled in only when it is asked for
    auto k = out.evaluated ? k_raster_fwd<CM, TW, TH, LIDAR, true> : k_raster_fwd<CM, TW, TH, LIDAR, false>;
    set_smem(k, sm);
    k<<<blocks, NT, sm, st>>>(fr, in, out);
}

template <int CM, int TW, int TH, bool LIDAR>
static void launch_bwd_t(const Frame& fr, int blocks, const RasterIn& in, const RasterGrad& g, bool recompute,
                         cudaStream_t st) {
    constexpr int NT = TW * TH / RaysPerThread<CM, true, LIDAR, TW * TH>::value;
    if constexpr (CM == 16 && !LIDAR && TW * TH == 256) {   // 16 channels on 256-ray tiles: tensor cores
        static_assert(NT == 64, "two warps of 4 rays per thread");
        constexpr int KB = 16;   // list positions per batch: 7 blocks of 2 warps per SM
        // lists of cameras without the tile cull hold entries dead in their tile: pack the
        // live ones at staging
        bool culled = true;
        for (int c = 0; c < fr.n_cams; c++) culled = culled && (fr.s[fr.cam_sensors[c]].support & 4);
        auto k = recompute ? (culled ? k_raster_bwd_cam16<TW, TH, true, KB, false> : k_raster_bwd_cam16<TW, TH, true, KB, true>)
                           : (culled ? k_raster_bwd_cam16<TW, TH, false, KB, false> : k_raster_bwd_cam16<TW, TH, false, KB, true>);
        const size_t bytes = recompute ? sizeof(cam16::Smem<KB, true>) : sizeof(cam16::Smem<KB, false>);
        set_smem(k, bytes);
        k<<<blocks, NT, bytes, st>>>(fr, in, g);
        return;
    }
    using LY = BwdLayout<CM, LIDAR>;
    const size_t sm = sizeof(Stage<CM, NT, LIDAR>) + sizeof(float) * LY::slices(NT / 32) * NT * LY::kRow;
    if (recompute) {
        auto k = k_raster_bwd<CM, TW, TH, LIDAR, true>;
        set_smem(k, sm);
        k<<<blocks, NT, sm, st>>>(fr, in, g);
    } else {
        auto k = k_raster_bwd<CM, TW, TH, LIDAR, false>;
        set_smem(k, sm);
        k<<<blocks, NT, sm, st>>>(fr, in, g);
    }
}

// Free-ray lists (App. A.2): one block per chunk of 256 rays whatever the lidar's tile
// shape (the tile only selects the Gaussian list); `blocks` bounds the number of chunks.
template <int CM>
bool dispatch_list(const Frame& fr, int blocks, const RasterIn& in, const RasterOut* out, const RasterGrad* g,
                   bool recompute, cudaStream_t st) {
    if (out) {
        constexpr int NT = 256 / RaysPerThread<CM, false, true, 256>::value;
        const size_t sm = sizeof(Stage<CM, NT, true>);
        auto k = k_raster_fwd<CM, 32, 8, true, false, true>;
        set_smem(k, sm);
        k<<<blocks, NT, sm, st>>>(fr, in, *out);
        return true;
    }
    constexpr int NT = 256 / RaysPerThread<CM, true, true, 256>::value;
    using LY = BwdLayout<CM, true>;
    const size_t sm = sizeof(Stage<CM, NT, true>) + sizeof(float) * LY::slices(NT / 32) * NT * LY::kRow;
    auto k = recompute ? k_raster_bwd<CM, 32, 8, true, true, true> : k_raster_bwd<CM, 32, 8, true, false, true>;
    set_smem(k, sm);
    k<<<blocks, NT, sm, st>>>(fr, in, *g);
    return true;
}

template <int CM, bool LIDAR>
bool dispatch_shape(int tw, int th, const Frame& fr, int blocks, const RasterIn& in, const RasterOut* out,
                    const RasterGrad* g, bool recompute, cudaStream_t st) {
#define SPLAT_SHAPE(W, H)                                                     \
    if (tw == W && th == H) {                                                 \
        if (out) launch_fwd_t<CM, W, H, LIDAR>(fr, blocks, in, *out, st);     \
        else launch_bwd_t<CM, W, H, LIDAR>(fr, blocks, in, *g, recompute, st); \
        return true;                                                          \
    }
    if constexpr (!LIDAR) {
        SPLAT_SHAPE(16, 16)
        SPLAT_SHAPE(8, 8)
        SPLAT_SHAPE(32, 8)
        SPLAT_SHAPE(16, 32)
    } else {
        SPLAT_SHAPE(32, 8)
        SPLAT_SHAPE(16, 8)
        SPLAT_SHAPE(32, 16)
        SPLAT_SHAPE(64, 8)
    }
#undef SPLAT_SHAPE
    return false;
}

#define SPLAT_INSTANTIATE_CM(CMV)                                                                              \
    template bool dispatch_shape<CMV, false>(int, int, const Frame&, int, const RasterIn&, const RasterOut*,  \
                                             const RasterGrad*, bool, cudaStream_t);                         \
    template bool dispatch_shape<CMV, true>(int, int, const Frame&, int, const RasterIn&, const RasterOut*,   \
                                            const RasterGrad*, bool, cudaStream_t);                          \
    template bool dispatch_list<CMV>(const Frame&, int, const RasterIn&, const RasterOut*, const RasterGrad*, \
                                     bool, cudaStream_t);

}  // namespace splat
