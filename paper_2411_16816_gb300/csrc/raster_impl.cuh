// raster.cu -- tile rasterization of cameras and lidars, forward and backward.
//
// Camera (paper Sec. 3.2 "Rasterization"): one CTA per tile, one thread per pixel, row
// time t_pix = ((row + 0.5) / H - 0.5) t_rs (+ time offset) (Eq. t_pix), Gaussians
// blended front to back (Eq. alpha blend) with the EWA-blurred alpha of Eq. (alpha) at the
// rolling-shutter shifted mean of Eq. (delta).
// Lidar (Sec. 3.3 "Rasterization", App. A.2): one CTA per lidar tile (N_phi azimuth bins x
// N_omega beams), one thread per ray with its own (phi, omega, t); the expected range
// blends r + v_r t and the median range is the rolling-shutter range of the first
// Gaussian after which the transmittance is below 0.5.  Threads without a ray (the
// ragged last azimuth column) only help stage Gaussians, as in App. A.2.
//
// Gaussians are staged through shared memory a batch of one-per-thread at a time; the
// block stops as soon as every thread is done (__syncthreads_count vote).
// The backward walks each tile's list back to front, rebuilding transmittance by
// division, sums each Gaussian's gradient over the warp's 32 rays with shuffles and
// issues one vector atomic per warp and Gaussian.  With `out_T`/`out_last` absent it first
// recomputes them for its tile (no per-pixel forward state kept).
#pragma once
#include "types.cuh"

namespace splat {

struct RayCtx {
    bool inside;
    float pa, pb, t;
    int64_t o;      // output index
    int s;          // sensor
    int gtile;
};

template <int TW, int TH, bool LIDAR>
__device__ __forceinline__ RayCtx ray_setup(const Frame& fr) {
    RayCtx r;
    r.s = sensor_of_block(fr, blockIdx.x, LIDAR);
    const SensorDev& S = fr.s[r.s];
    const int lt = blockIdx.x - S.block_base;
    const int tx = lt % S.tiles_x, ty = lt / S.tiles_x;
    r.gtile = S.tile_base + lt;
    const int lx = threadIdx.x % TW, ly = threadIdx.x / TW;
    if (!LIDAR) {
        const int col = tx * TW + lx, row = ty * TH + ly;
        r.inside = col < S.width && row < S.height;
        r.pa = col + 0.5f;
        r.pb = row + 0.5f;
        r.t = ((row + 0.5f) / (float)S.height - 0.5f) * S.rs + S.dt;
        r.o = (int64_t)S.ray_base + (int64_t)row * S.width + col;
    } else {
        const int a = tx * TW + lx, b = ty * TH + ly;
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

template <int CM, int B, bool LIDAR>
struct Stage {
    float4 g0[B];
    float4 g1[B];
    float2 g2[LIDAR ? B : 1];
    uint32_t id[B];
    alignas(16) float f[B * CM];
};

template <int CM, int B, bool LIDAR>
__device__ __forceinline__ void stage_load(Stage<CM, B, LIDAR>& sm, const RasterIn& in, int s, int64_t j, int slot) {
    const uint32_t id = in.ids[j];
    sm.id[slot] = id;
    sm.g0[slot] = in.rec[rec_index(s, 0, in.n, id)];
    sm.g1[slot] = in.rec[rec_index(s, 1, in.n, id)];
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

// alpha of one staged Gaussian at the ray; returns false if it is skipped.
template <bool LIDAR>
__device__ __forceinline__ bool eval_alpha(const float4 g0, const float4 g1, const RayCtx& r, float& dx, float& dy,
                                           float& G, float& alpha, bool& clamped) {
    dx = r.pa - (g0.x + g0.z * r.t);
    dy = r.pb - (g0.y + g0.w * r.t);
    if (LIDAR) dx = wrap_pi(dx);
    const float sig = 0.5f * (g1.x * dx * dx + g1.z * dy * dy) + g1.y * dx * dy;
    if (sig < 0.f) return false;
    G = __expf(-sig);
    const float a = g1.w * G;
    clamped = a > kAlphaMax;
    alpha = clamped ? kAlphaMax : a;
    return alpha >= kAlphaMin;
}

struct FwdState {
    float T;
    int last;
    int evals;   // list entries examined (blended, skipped or terminating)
    float de, dm;
    bool med, done;
};

// Front-to-back blend of the tile's list for this thread's ray.  F may be null when
// only the transmittance and the last index are wanted (recomputation).
template <int CM, int B, bool LIDAR, bool WANT_F>
__device__ __forceinline__ void forward_tile(Stage<CM, B, LIDAR>& sm, const RasterIn& in, const RayCtx& r, int2 range,
                                             FwdState& st, float* F) {
    st.T = 1.f;
    st.last = 0;
    st.evals = 0;
    st.de = 0.f;
    st.dm = 0.f;
    st.med = false;
    st.done = !r.inside;
    for (int start = range.x; start < range.y; start += B) {
        if (__syncthreads_count(st.done) == B) break;
        const int j = start + threadIdx.x;
        if (j < range.y) stage_load<CM, B, LIDAR>(sm, in, r.s, j, threadIdx.x);
        __syncthreads();
        if (!st.done) {
            const int nb = min(B, range.y - start);
            for (int k = 0; k < nb; k++) {
                float dx, dy, G, a;
                bool cl;
                st.evals++;
                if (!eval_alpha<LIDAR>(sm.g0[k], sm.g1[k], r, dx, dy, G, a, cl)) continue;
                const float Tn = st.T * (1.f - a);
                if (Tn < kTEps) {
                    st.done = true;
                    break;
                }
                const float wgt = a * st.T;
                if (WANT_F) {
#pragma unroll
                    for (int c = 0; c < CM; c++) F[c] += sm.f[k * CM + c] * wgt;
                }
                if (LIDAR) {
                    const float rrs = sm.g2[k].x + sm.g2[k].y * r.t;
                    st.de += rrs * wgt;
                    if (!st.med && Tn < 0.5f) {
                        st.dm = rrs;
                        st.med = true;
                    }
                }
                st.T = Tn;
                st.last = start + k - range.x + 1;
            }
        }
    }
}

template <int CM, int TW, int TH, bool LIDAR>
__global__ void __launch_bounds__(TW* TH) k_raster_fwd(const __grid_constant__ Frame fr, RasterIn in, RasterOut out) {
    constexpr int B = TW * TH;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Stage<CM, B, LIDAR>& sm = *reinterpret_cast<Stage<CM, B, LIDAR>*>(smem_raw);
    const RayCtx r = ray_setup<TW, TH, LIDAR>(fr);
    const int2 range = in.ranges[r.gtile];
    float F[CM];
#pragma unroll
    for (int c = 0; c < CM; c++) F[c] = 0.f;
    FwdState st;
    forward_tile<CM, B, LIDAR, true>(sm, in, r, range, st, F);
    if (out.evaluated) {
        unsigned long long e = (unsigned long long)st.evals;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(out.evaluated, e);
    }
    if (!r.inside) return;
    const int C = in.C;
    float* fo = out.feat + r.o * C;
    if ((C & 3) == 0) {
#pragma unroll
        for (int c = 0; c < CM; c += 4)
            if (c < C) *reinterpret_cast<float4*>(fo + c) = make_float4(F[c], F[c + 1], F[c + 2], F[c + 3]);
    } else {
#pragma unroll
        for (int c = 0; c < CM; c++)
            if (c < C) fo[c] = F[c];
    }
    if (out.T) out.T[r.o] = st.T;
    if (out.last) out.last[r.o] = st.last;
    if (LIDAR) {
        out.range_exp[r.o] = st.de;
        if (out.range_med) out.range_med[r.o] = st.dm;
        out.alpha[r.o] = 1.f - st.T;
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int CM, int TW, int TH, bool LIDAR, bool RECOMPUTE>
__global__ void __launch_bounds__(TW* TH) k_raster_bwd(const __grid_constant__ Frame fr, RasterIn in, RasterGrad gr) {
    constexpr int B = TW * TH;
    constexpr int C = CM;   // register arrays sized by the maximum; lanes beyond in.C stay zero
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Stage<CM, B, LIDAR>& sm = *reinterpret_cast<Stage<CM, B, LIDAR>*>(smem_raw);
    __shared__ int s_max_last[B / 32];
    const int Crt = in.C;
    const RayCtx r = ray_setup<TW, TH, LIDAR>(fr);
    const int2 range = in.ranges[r.gtile];
    float Tfin;
    int last;
    if (RECOMPUTE) {
        FwdState st;
        forward_tile<CM, B, LIDAR, false>(sm, in, r, range, st, nullptr);
        Tfin = st.T;
        last = st.last;
    } else {
        Tfin = r.inside ? gr.T[r.o] : 1.f;
        last = r.inside ? gr.last[r.o] : 0;
    }
    float gF[C], Bc[C];
    float gT = 0.f, gD = 0.f;
    if (r.inside) {
#pragma unroll
        for (int c = 0; c < C; c++) gF[c] = c < Crt ? gr.dfeat[r.o * Crt + c] : 0.f;
        if (!LIDAR) {
            gT = gr.dT ? gr.dT[r.o] : 0.f;
        } else {
            gT = gr.dalpha ? -gr.dalpha[r.o] : 0.f;
            gD = gr.drange ? gr.drange[r.o] : 0.f;
        }
    } else {
#pragma unroll
        for (int c = 0; c < C; c++) gF[c] = 0.f;
    }
#pragma unroll
    for (int c = 0; c < C; c++) Bc[c] = 0.f;
    float BD = 0.f;
    // tile-wide maximum of the last blended index
    const int wl = __reduce_max_sync(0xffffffffu, (unsigned)last);
    if ((threadIdx.x & 31) == 0) s_max_last[threadIdx.x >> 5] = wl;
    __syncthreads();
    int max_last = 0;
#pragma unroll
    for (int w = 0; w < B / 32; w++) max_last = max(max_last, s_max_last[w]);
    max_last = min(max_last, range.y - range.x);   // never walk past this tile's list
    last = min(last, range.y - range.x);
    float T = Tfin;
    const int lane = threadIdx.x & 31;
    float4* gp0 = gr.grad_proj + rec_index(r.s, 0, in.n, 0);
    float4* gp1 = gr.grad_proj + rec_index(r.s, 1, in.n, 0);
    float4* gp2 = gr.grad_proj + rec_index(r.s, 2, in.n, 0);
    for (int end = range.x + max_last; end > range.x; end -= B) {
        const int cnt = min(B, end - range.x);
        __syncthreads();
        if (threadIdx.x < cnt) stage_load<CM, B, LIDAR>(sm, in, r.s, end - 1 - threadIdx.x, threadIdx.x);
        __syncthreads();
        for (int k = 0; k < cnt; k++) {
            const int idx = end - 1 - k - range.x;
            float dx = 0.f, dy = 0.f, G = 0.f, a = 0.f;
            bool cl = false;
            bool contrib = r.inside && idx < last;
            if (contrib) contrib = eval_alpha<LIDAR>(sm.g0[k], sm.g1[k], r, dx, dy, G, a, cl);
            if (!__any_sync(0xffffffffu, contrib)) continue;
            float v[10 + C];
#pragma unroll
            for (int q = 0; q < 10 + C; q++) v[q] = 0.f;
            if (contrib) {
                const float Ti = T / (1.f - a);
                const float wgt = a * Ti;
                float dot = 0.f;
#pragma unroll
                for (int c = 0; c < C; c++) {
                    const float f = sm.f[k * CM + c];
                    v[10 + c] = wgt * gF[c];
                    dot += gF[c] * (f - Bc[c]);
                    Bc[c] = f * a + (1.f - a) * Bc[c];
                }
                float dalpha = Ti * dot - gT * Tfin / (1.f - a);
                if (LIDAR) {
                    const float rrs = sm.g2[k].x + sm.g2[k].y * r.t;
                    dalpha += Ti * gD * (rrs - BD);
                    BD = rrs * a + (1.f - a) * BD;
                    const float drrs = gD * wgt;
                    v[8] = drrs;          // d range
                    v[9] = drrs * r.t;    // d v_r
                }
                if (!cl) {
                    const float4 g1 = sm.g1[k];
                    const float dsig = -dalpha * a;
                    v[7] = dalpha * G;                        // d o'
                    v[4] = dsig * 0.5f * dx * dx;              // d conic a
                    v[5] = dsig * dx * dy;                     // d conic b
                    v[6] = dsig * 0.5f * dy * dy;              // d conic c
                    const float ddx = dsig * (g1.x * dx + g1.y * dy);
                    const float ddy = dsig * (g1.y * dx + g1.z * dy);
                    v[0] = -ddx;                               // d mean a
                    v[1] = -ddy;                               // d mean b
                    v[2] = -ddx * r.t;                         // d v_a
                    v[3] = -ddy * r.t;                         // d v_b
                }
                T = Ti;
            }
#pragma unroll
            for (int q = 0; q < 10 + C; q++) {
                if (!LIDAR && (q == 8 || q == 9)) continue;
                if (q >= 10 + Crt) continue;
                v[q] = warp_sum(v[q]);
            }
            if (lane == 0) {
                const uint32_t id = sm.id[k];
                atomicAdd(gp0 + id, make_float4(v[0], v[1], v[2], v[3]));
                atomicAdd(gp1 + id, make_float4(v[4], v[5], v[6], v[7]));
                if (LIDAR) atomicAdd(reinterpret_cast<float2*>(gp2 + id), make_float2(v[8], v[9]));
                float* df = gr.dfeatures + (int64_t)id * Crt;
                if ((Crt & 3) == 0) {
#pragma unroll
                    for (int c = 0; c < C; c += 4)
                        if (c < Crt)
                            atomicAdd(reinterpret_cast<float4*>(df + c),
                                      make_float4(v[10 + c], v[11 + c], v[12 + c], v[13 + c]));
                } else {
#pragma unroll
                    for (int c = 0; c < C; c++)
                        if (c < Crt) atomicAdd(df + c, v[10 + c]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------
// Host launch helpers (instantiated per channel bucket in raster_c*.cu)
// ---------------------------------------------------------------------------------

template <typename K>
static void set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int CM, int TW, int TH, bool LIDAR>
static void launch_fwd_t(const Frame& fr, int blocks, const RasterIn& in, const RasterOut& out, cudaStream_t st) {
    const size_t sm = sizeof(Stage<CM, TW * TH, LIDAR>);
    auto k = k_raster_fwd<CM, TW, TH, LIDAR>;
    set_smem(k, sm);
    k<<<blocks, TW * TH, sm, st>>>(fr, in, out);
}

template <int CM, int TW, int TH, bool LIDAR>
static void launch_bwd_t(const Frame& fr, int blocks, const RasterIn& in, const RasterGrad& g, bool recompute,
                         cudaStream_t st) {
    const size_t sm = sizeof(Stage<CM, TW * TH, LIDAR>);
    if (recompute) {
        auto k = k_raster_bwd<CM, TW, TH, LIDAR, true>;
        set_smem(k, sm);
        k<<<blocks, TW * TH, sm, st>>>(fr, in, g);
    } else {
        auto k = k_raster_bwd<CM, TW, TH, LIDAR, false>;
        set_smem(k, sm);
        k<<<blocks, TW * TH, sm, st>>>(fr, in, g);
    }
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
                                            const RasterGrad*, bool, cudaStream_t);

}  // namespace splat
