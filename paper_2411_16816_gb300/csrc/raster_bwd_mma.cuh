// raster_bwd_mma.cuh -- camera backward for the 16-channel bucket on 256-ray tiles, with
// the two feature contractions of the blend's reverse mode on the tensor cores.
//
// Reverse mode of the front-to-back blend (Eq. alpha blend, Sec. 3.2), per ray r and list
// entry e taken back to front, g_r the upstream gradient of the ray's features, T_e the
// transmittance in front of e and S_e the normalised blend of everything behind it:
//   dL/dalpha_e = T_e (f_e . g_r - S_e) / (1 - alpha_e) - dL/dT_final T_final / (1 - alpha_e)
//   dL/df_e    += w_e,r g_r,   w_e,r = alpha_e T_e.
// Both products over the channels are dense contractions of a group of entries with the
// rays of a warp: P = F G^T (entries x rays, K = 16 channels) and dF = W G (entries x
// channels, K = the warp's 128 rays).  Each warp forms them per group of 8 staged entries
// with mma.sync m16n8k16 on split BF16 operands (x = hi + lo, hi = bf16(x), lo = bf16(x -
// hi); the products hi.hi + hi.lo + lo.hi accumulate in FP32, about 2^-16 relative per
// term).  The per-ray chain (alpha, transmittance, suffix sum, 8 geometric moments and
// their warp sums) stays on the CUDA cores, reads P from shared memory and writes the
// blend weights back in place; the upstream gradients live in shared memory (BF16 high
// parts and residuals) instead of 64 registers per thread.
//
// The two warps of a tile run independently: each stages the entries its own rays reach
// (16 list positions per batch, deepest first; for lists of uncut cameras only the
// entries live in the tile, packed), forms its sums and flushes them with its own float4
// atomics.  The chain sums the moments of Pn dx and Pn dy (Pn = -dL/dsigma); the flush
// turns them into the mean gradients with the entry's conic, -ddx = Pn (a dx + b dy),
// -ddy = Pn (b dx + c dy).  The staged conic is (a/2, b, c/2), as the evaluation uses it.
#pragma once

#include "mma.cuh"

namespace splat {
namespace cam16 {

constexpr int kG = 8;       // entries per MMA group
constexpr int kRowW = 68;   // 32-bit words per P/W row: 256 B + 16 B (conflict-free stores and ldmatrix rows)
constexpr int kRow = 24;    // accumulator row: 8 geometric sums, then 16 feature sums

// Each warp owns 128 rays, lane l the rays rho = 4 l + q (q = the thread's ray index).
// Its P/W rows: row e (entry e of the group) first holds P of every lane's rays 0 and 1,
// then the blend weights' BF16 high parts of all 128 rays in rho order; row 8 + e holds P
// of rays 2 and 3, then the residuals.  A lane reads and overwrites only its own 8 bytes
// of each row.
template <int KB>
struct BwdArea {
    Stage<16, KB, false> st[2];   // per warp; st.f holds the features as BF16: KB x 16 high parts, then residuals
    float acc[2][KB][kRow];       // per warp: the batch's per-entry sums
};
template <int KB, bool RECOMPUTE>
struct Smem {
    union {
        BwdArea<KB> b;
        Stage<16, RECOMPUTE ? 64 : 1, false> fwd;   // the recomputation's forward pass, before the backward
    } u;
    alignas(16) uint32_t pw[2][16 * kRowW];
    alignas(16) uint4 gh[2][256];      // per warp: upstream gradients, high parts, rho x 2 chunks of 8 channels
    alignas(16) uint4 gl[2][256];      // residuals
};

// Chunk (rho, cb) of a warp's gradient plane, swizzled within its 128-byte group so that
// the eight rows of every ldmatrix, in either operand layout, fall in distinct banks.
__device__ __forceinline__ int gchunk(int rho, int cb) { return (2 * rho + cb) ^ ((rho >> 2) & 7); }

// The 16 features of Gaussian `id` (zero past the channel count).
__device__ __forceinline__ void load_feat16(const RasterIn& in, uint32_t id, float (&f)[16]) {
    const int C = in.C;
    const float* fp = in.feat + (int64_t)id * C;
    if ((C & 3) == 0) {
#pragma unroll
        for (int c = 0; c < 16; c += 4) {
            const float4 v = c < C ? *reinterpret_cast<const float4*>(fp + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            f[c] = v.x;
            f[c + 1] = v.y;
            f[c + 2] = v.z;
            f[c + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int c = 0; c < 16; c++) f[c] = c < C ? fp[c] : 0.f;
    }
}

// Stages a live list entry (its Gaussian `id`, records g0 g1, features f, list position
// `pos`) at its packed slot: the records, id, position and split features.
template <int KB>
__device__ __forceinline__ void stage_live(Stage<16, KB, false>& st, uint32_t id, float4 g0, float4 g1,
                                           const float (&f)[16], int slot, int pos) {
    st.id[slot] = id;
    st.g0[slot] = g0;
    st.g1[slot] = make_float4(__fmul_rn(0.5f, g1.x), g1.y, __fmul_rn(0.5f, g1.z), g1.w);   // half conic (exact)
    st.live[slot] = pos;   // the backward keeps list positions here
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int p = 0; p < 8; p++) split_pair(f[2 * p], f[2 * p + 1], hi[p], lo[p]);
    uint4* fh = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(st.f) + slot * 16);
    uint4* fl = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(st.f) + KB * 16 + slot * 16);
    fh[0] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    fh[1] = make_uint4(hi[4], hi[5], hi[6], hi[7]);
    fl[0] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    fl[1] = make_uint4(lo[4], lo[5], lo[6], lo[7]);
}

// Clears a slot past the batch's live entries: zero records and features, so that every
// term of the chain is finite and zero for it.
template <int KB>
__device__ __forceinline__ void stage_empty(Stage<16, KB, false>& st, int slot) {
    st.g0[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    st.g1[slot] = make_float4(0.f, 0.f, 0.f, 0.f);
    st.live[slot] = 0;
    uint4* fh = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(st.f) + slot * 16);
    uint4* fl = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(st.f) + KB * 16 + slot * 16);
    fh[0] = fh[1] = fl[0] = fl[1] = make_uint4(0u, 0u, 0u, 0u);
}

// Stages list entry j at `slot` without packing (lists of culled cameras, where almost
// every entry is live): records, id, live flag, split features; a slot past the batch
// gets zero records and features and is marked dead.
template <int KB>
__device__ __forceinline__ void stage_entry(Stage<16, KB, false>& st, const RasterIn& in, int s, int64_t j, int slot,
                                            bool valid, const TileBox& box) {
    if (!valid) {
        stage_empty<KB>(st, slot);
        return;
    }
    const uint32_t id = load_id(in, j);
    const float4 g0 = in.rec[rec_index(s, 0, in.n, id)];
    const float4 g1 = in.rec[rec_index(s, 1, in.n, id)];
    float f[16];
    load_feat16(in, id, f);
    stage_live<KB>(st, id, g0, g1, f, slot, 0);
    st.live[slot] = tile_live(g0, g1, box);
}

}  // namespace cam16

// One block per 256-ray camera tile, 2 warps, 4 rays per thread (pixel threadIdx.x + 64 q);
// KB list positions per batch and warp.  COMPACT packs the live entries of each batch (for
// lists that hold entries dead in their tile); otherwise every position is staged with a
// live flag.
template <int TW, int TH, bool RECOMPUTE, int KB, bool COMPACT>
__global__ void __launch_bounds__(64, 7)
    k_raster_bwd_cam16(const __grid_constant__ Frame fr, RasterIn in, RasterGrad gr) {
    using namespace cam16;
    constexpr int PX = 4, NT = 64;
    static_assert(TW * TH == PX * NT, "256-ray tiles");
    static_assert(KB % kG == 0 && KB <= NT, "whole groups, one staging thread per entry");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<KB, RECOMPUTE>& s = *reinterpret_cast<Smem<KB, RECOMPUTE>*>(smem_raw);
    TileCtx tc;
    RayCtx r[PX];
    if (!block_setup<TW, TH, false, false, PX, NT>(fr, in, tc, r)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float2 rpa[2], rpb[2], rt[2];   // ray pairs (0, 1) and (2, 3)
#pragma unroll
    for (int qp = 0; qp < 2; qp++) {
        rpa[qp] = make_float2(r[2 * qp].pa, r[2 * qp + 1].pa);
        rpb[qp] = make_float2(r[2 * qp].pb, r[2 * qp + 1].pb);
        rt[qp] = make_float2(r[2 * qp].t, r[2 * qp + 1].t);
    }
    const int2 range = load_range(in, tc.gtile);
    const int len = range.y - range.x;
    const TileBox box = camera_tile_box(fr.s[tc.s], tc.tx, tc.ty, TW, TH);
    float Tfin[PX];
    int last[PX];
    if constexpr (RECOMPUTE) {
        FwdState st[PX];
        forward_tile<16, TW, TH, false, PX, false>(s.u.fwd, in, tc, box, r, range, st, nullptr);
#pragma unroll
        for (int q = 0; q < PX; q++) {
            Tfin[q] = st[q].T;
            last[q] = min(st[q].last, len);
        }
        __syncthreads();   // the forward's staging area becomes the accumulators
    } else {
#pragma unroll
        for (int q = 0; q < PX; q++) {
            Tfin[q] = r[q].inside ? gr.T[r[q].o] : 1.f;
            last[q] = r[q].inside ? min(gr.last[r[q].o], len) : 0;   // never past this tile's list
        }
    }
    for (int i = lane; i < KB * kRow; i += 32) (&s.u.b.acc[w][0][0])[i] = 0.f;
    // this warp's upstream feature gradients, split, into its planes (ray rho = 4 lane + q)
    const int C = in.C;
    float gTT[PX], T[PX], S[PX];
    int my_last = 0;
#pragma unroll
    for (int q = 0; q < PX; q++) {
        float gv[16];
#pragma unroll
        for (int c = 0; c < 16; c++) gv[c] = (r[q].inside && c < C) ? gr.dfeat[r[q].o * C + c] : 0.f;
        uint32_t hi[8], lo[8];
#pragma unroll
        for (int p = 0; p < 8; p++) split_pair(gv[2 * p], gv[2 * p + 1], hi[p], lo[p]);
        const int rho = 4 * lane + q;
        s.gh[w][gchunk(rho, 0)] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        s.gh[w][gchunk(rho, 1)] = make_uint4(hi[4], hi[5], hi[6], hi[7]);
        s.gl[w][gchunk(rho, 0)] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        s.gl[w][gchunk(rho, 1)] = make_uint4(lo[4], lo[5], lo[6], lo[7]);
        const float gT = (r[q].inside && gr.dT) ? gr.dT[r[q].o] : 0.f;
        gTT[q] = gT * Tfin[q];
        T[q] = Tfin[q];
        S[q] = 0.f;   // sum_c g_c B_c, B = normalised blend of everything behind
        my_last = max(my_last, last[q]);
    }
    const int wl = __reduce_max_sync(0xffffffffu, (unsigned)my_last);   // this warp's deepest entry
    __syncwarp();
    float4* gp0 = gr.grad_proj + rec_index(tc.s, 0, in.n, 0);
    float4* gp1 = gr.grad_proj + rec_index(tc.s, 1, in.n, 0);
    Stage<16, KB, false>& sw = s.u.b.st[w];   // this warp's staging area
    const bf16* Fh = reinterpret_cast<const bf16*>(sw.f);
    const bf16* Fl = Fh + KB * 16;
    uint32_t* pw = s.pw[w];
    const int g = lane >> 2, t = lane & 3, mi = lane >> 3, ri = lane & 7;   // fragment / ldmatrix roles
    float dtime = 0.f;   // this thread's share of dL/d (camera time offset)
    // The two warps of a tile run independently: each stages the entries its rays reach
    // (from its own deepest entry up), forms its sums and flushes them, with no barrier.
    for (int end = range.x + wl; end > range.x; end -= KB) {
        const int cnt = min(KB, end - range.x);
        // the batch's list positions [end - cnt, end), deepest first: only the entries that can
        // reach alpha >= 1/255 somewhere in the tile are staged, packed in that order, each
        // with its list position
        __syncwarp();
        int n_live = cnt;   // staged slots
        if constexpr (COMPACT) {
            const int j = end - 1 - lane;
            uint32_t id = 0;
            float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
            bool lv = false;
            if (lane < cnt) {
                id = load_id(in, j);
                g0 = in.rec[rec_index(tc.s, 0, in.n, id)];
                g1 = in.rec[rec_index(tc.s, 1, in.n, id)];
                lv = tile_live(g0, g1, box);
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, lv);
            n_live = __popc(bal);
            if (lv) {
                float f[16];
                load_feat16(in, id, f);
                stage_live<KB>(sw, id, g0, g1, f, __popc(bal & ((1u << lane) - 1u)), j - range.x);
            }
            if (lane >= n_live && lane < KB) stage_empty<KB>(sw, lane);
        } else {
            if (lane < KB) stage_entry<KB>(sw, in, tc.s, end - 1 - lane, lane, lane < cnt, box);
        }
        __syncwarp();
        for (int k0 = 0; k0 < n_live; k0 += kG) {
            const int n = min(kG, n_live - k0);
            // the group's shallowest entry is its last
            const int shallow = COMPACT ? sw.live[k0 + n - 1] : end - 1 - (k0 + n - 1) - range.x;
            if (shallow >= wl) continue;   // every entry deeper than this warp's rays reach
            // ---- P = F G^T: rows of the MMA are rays, columns the group's entries ----
            __syncwarp();
            uint32_t bF[4];   // B fragments: F high (k 0-7, 8-15), F residual (k 0-7, 8-15)
            ldsm_x4(bF, (mi < 2 ? Fh : Fl) + (k0 + ri) * 16 + (mi & 1) * 8);
#pragma unroll
            for (int j = 0; j < 8; j++) {
                // A rows of m-tile j: row ri + 8 h' is ray 16 j + 4 (ri & 3) + 2 (ri >> 2) + h', so that
                // rows g and g + 8 of the result are a lane's consecutive ray pair
                const int rho = 16 * j + 4 * (ri & 3) + 2 * (ri >> 2) + (mi & 1);
                uint32_t aH[4], aL[4];
                ldsm_x4(aH, &s.gh[w][gchunk(rho, mi >> 1)]);
                ldsm_x4(aL, &s.gl[w][gchunk(rho, mi >> 1)]);
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                mma16816(c, aH, bF[0], bF[1]);
                mma16816(c, aH, bF[2], bF[3]);
                mma16816(c, aL, bF[0], bF[1]);
                // c: (ray pair of lane 4 j + (g & 3), pair g >> 2) x (entries 2 t, 2 t + 1)
                const int slot = 4 * j + (g & 3), hh = g >> 2;
                *reinterpret_cast<float2*>(pw + (2 * t + 8 * hh) * kRowW + 2 * slot) = make_float2(c[0], c[2]);
                *reinterpret_cast<float2*>(pw + (2 * t + 1 + 8 * hh) * kRowW + 2 * slot) = make_float2(c[1], c[3]);
            }
            __syncwarp();
            // ---- the rays' chains, entry by entry, back to front ----
            // Without branches: an entry past the group's staged entries, deeper than every
            // ray of the warp or dead in the tile takes alpha = 0 for every ray, which leaves T
            // and S bit for bit unchanged and writes zero weights and sums.
#pragma unroll 1
            for (int e2 = 0; e2 < kG; e2 += 2) {   // two entries, then their warp sums
                if (e2 >= n) {   // past the group's live entries (warp-uniform): zero weights
                    *reinterpret_cast<uint2*>(pw + e2 * kRowW + 2 * lane) = make_uint2(0u, 0u);
                    *reinterpret_cast<uint2*>(pw + (e2 + 8) * kRowW + 2 * lane) = make_uint2(0u, 0u);
                    *reinterpret_cast<uint2*>(pw + (e2 + 1) * kRowW + 2 * lane) = make_uint2(0u, 0u);
                    *reinterpret_cast<uint2*>(pw + (e2 + 9) * kRowW + 2 * lane) = make_uint2(0u, 0u);
                    continue;
                }
                float vv[16];                        // the two entries' 8 geometric values
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const int e = e2 + u;
                    uint2* wa = reinterpret_cast<uint2*>(pw + e * kRowW + 2 * lane);
                    uint2* wb = reinterpret_cast<uint2*>(pw + (e + 8) * kRowW + 2 * lane);
                    const int k = k0 + e;
                    const int idx = COMPACT ? sw.live[k] : end - 1 - k - range.x;   // list position
                    const bool act = e < n && idx < wl && (COMPACT || sw.live[k]);
                    const float4 g0 = sw.g0[k], g1 = sw.g1[k];
                    float2 dx2[2], dy2[2], G2[2], a2[2];
                    bool on[PX], cl[PX];
#pragma unroll
                    for (int qp = 0; qp < 2; qp++) {
                        float2 sig2, au2;
                        eval_alpha2<false, true>(g0, g1, rpa[qp], rpb[qp], rt[qp], sig2, a2[qp], dx2[qp], dy2[qp], G2[qp],
                                                 au2);
                        on[2 * qp] = act && sig2.x >= 0.f && a2[qp].x >= kAlphaMin && idx < last[2 * qp];
                        on[2 * qp + 1] = act && sig2.y >= 0.f && a2[qp].y >= kAlphaMin && idx < last[2 * qp + 1];
                        cl[2 * qp] = au2.x > kAlphaMax;
                        cl[2 * qp + 1] = au2.y > kAlphaMax;
                    }
                    const float2 Pa = *reinterpret_cast<const float2*>(wa), Pb = *reinterpret_cast<const float2*>(wb);
                    const float2 m1 = make_float2(-1.f, -1.f);
                    float2 acc[8];
                    uint32_t whi[2], wlo[2];
#pragma unroll
                    for (int qp = 0; qp < 2; qp++) {
                        const int q0 = 2 * qp, q1 = 2 * qp + 1;
                        // a ray that does not blend this Gaussian gets alpha = 0: every term vanishes
                        const float2 aq = make_float2(on[q0] ? a2[qp].x : 0.f, on[q1] ? a2[qp].y : 0.f);
                        const float2 Gq = make_float2(on[q0] ? G2[qp].x : 0.f, on[q1] ? G2[qp].y : 0.f);
                        const float2 om = __ffma2_rn(aq, m1, make_float2(1.f, 1.f));
                        const float2 inv = make_float2(rcp_approx(om.x), rcp_approx(om.y));
                        const float2 Ti = __fmul2_rn(make_float2(T[q0], T[q1]), inv);
                        const float2 wgt = __fmul2_rn(aq, Ti);
                        const float2 Gf = qp == 0 ? Pa : Pb;   // sum_c g_c f_c of the pair
                        const float2 S2 = make_float2(S[q0], S[q1]);
                        const float2 dS = __ffma2_rn(S2, m1, Gf);   // Gf - S
                        const float2 dal = __ffma2_rn(Ti, dS, __fmul2_rn(make_float2(-gTT[q0], -gTT[q1]), inv));
                        const float2 Sn = __ffma2_rn(aq, dS, S2);
                        S[q0] = Sn.x;
                        S[q1] = Sn.y;
                        // clamped alpha (o' G > 0.999) passes no gradient to o' and the exponent
                        const float2 dg = make_float2((on[q0] && !cl[q0]) ? dal.x : 0.f, (on[q1] && !cl[q1]) ? dal.y : 0.f);
                        const float2 Pn = __fmul2_rn(dg, aq);   // -dL/dsigma
                        // the conic is the entry's own: -ddx = Pn (a dx + b dy), -ddy = Pn (b dx + c dy)
                        // are formed from the sums of Pn dx and Pn dy when the entry is flushed
                        const float2 hx = __fmul2_rn(Pn, dx2[qp]), hy = __fmul2_rn(Pn, dy2[qp]);
                        const float2 tq = rt[qp];
                        if (qp == 0) {
                            acc[0] = hx;
                            acc[1] = hy;
                            acc[2] = __fmul2_rn(hx, tq);
                            acc[3] = __fmul2_rn(hy, tq);
                            acc[4] = __fmul2_rn(hx, dx2[qp]);
                            acc[5] = __fmul2_rn(hx, dy2[qp]);
                            acc[6] = __fmul2_rn(hy, dy2[qp]);
                            acc[7] = __fmul2_rn(dg, Gq);
                        } else {
                            acc[0] = __fadd2_rn(acc[0], hx);
                            acc[1] = __fadd2_rn(acc[1], hy);
                            acc[2] = __ffma2_rn(hx, tq, acc[2]);
                            acc[3] = __ffma2_rn(hy, tq, acc[3]);
                            acc[4] = __ffma2_rn(hx, dx2[qp], acc[4]);
                            acc[5] = __ffma2_rn(hx, dy2[qp], acc[5]);
                            acc[6] = __ffma2_rn(hy, dy2[qp], acc[6]);
                            acc[7] = __ffma2_rn(dg, Gq, acc[7]);
                        }
                        split_pair(wgt.x, wgt.y, whi[qp], wlo[qp]);
                        T[q0] = Ti.x;
                        T[q1] = Ti.y;
                    }
                    *wa = make_uint2(whi[0], whi[1]);   // this lane's 4 weights: high parts, then residuals
                    *wb = make_uint2(wlo[0], wlo[1]);
                    // (Pn dx, Pn dy, Pn dx t, Pn dy t, Pn dx^2, Pn dx dy, Pn dy^2, dg G) summed over
                    // this thread's rays (Pn = -dL/dsigma); the flush turns them into gradients
                    float v[8];
#pragma unroll
                    for (int j = 0; j < 8; j++) v[j] = acc[j].x + acc[j].y;
                    // every pixel time carries the camera time offset; the mean moves by v t:
                    // dL/dt += -ddx vx - ddy vy = v0 (a vx + b vy) + v1 (b vx + c vy)
                    if (gr.dsensor)   // g1 holds (a/2, b, c/2, o')
                        dtime += v[0] * (2.f * g1.x * g0.z + g1.y * g0.w) + v[1] * (g1.y * g0.z + 2.f * g1.z * g0.w);
#pragma unroll
                    for (int j = 0; j < 8; j++) vv[8 * u + j] = v[j];
                }
                // warp sums of the 16 values: four halving steps (lane bits 4, 3, 2, 1) and one
                // whole sum; value (lane >> 1) & 15 -- entry (lane >> 4) & 1, term (lane >> 1) & 7 --
                // is reported by the even lanes
                halve_step<8>(vv, lane, 16);
                halve_step<4>(vv, lane, 8);
                halve_step<2>(vv, lane, 4);
                halve_step<1>(vv, lane, 2);
                vv[0] += __shfl_xor_sync(0xffffffffu, vv[0], 1);
                if ((lane & 1) == 0) s.u.b.acc[w][k0 + e2 + ((lane >> 4) & 1)][(lane >> 1) & 7] = vv[0];
            }
            __syncwarp();
            // ---- dF = W G: rows of the MMA are channels, columns the group's entries ----
            // one accumulator per product
            float d[3][4] = {};
#pragma unroll
            for (int k2 = 0; k2 < 8; k2++) {   // 16 rays per step
                const int rho = 16 * k2 + ri + 8 * (mi >> 1);
                uint32_t aH[4], aL[4], bW[4];
                ldsm_x4_trans(aH, &s.gh[w][gchunk(rho, mi & 1)]);
                ldsm_x4_trans(aL, &s.gl[w][gchunk(rho, mi & 1)]);
                // B fragments: weights' high parts (rays 16 k2 + 0-7, 8-15), residuals (the same)
                ldsm_x4(bW, pw + (ri + 8 * (mi >> 1)) * kRowW + 8 * k2 + 4 * (mi & 1));
                mma16816(d[0], aH, bW[0], bW[1]);
                mma16816(d[1], aL, bW[0], bW[1]);
                mma16816(d[2], aH, bW[2], bW[3]);
            }
#pragma unroll
            for (int i = 0; i < 4; i++) d[0][i] = (d[0][i] + d[1][i]) + d[2][i];
            // d: (channel g, entry 2 t), (g, 2 t + 1), (g + 8, 2 t), (g + 8, 2 t + 1)
            float* a0 = s.u.b.acc[w][k0 + 2 * t];
            float* a1 = s.u.b.acc[w][k0 + 2 * t + 1];
            a0[8 + g] = d[0][0];
            a1[8 + g] = d[0][1];
            a0[16 + g] = d[0][2];
            a1[16 + g] = d[0][3];
        }
        __syncwarp();
        // one set of vector atomics per (warp, Gaussian): flush this batch's sums
        if (lane < n_live) {
            const int slot = lane;
            float* a_row = s.u.b.acc[w][slot];
            const uint32_t id = sw.id[slot];
            const float4 q0 = *reinterpret_cast<float4*>(a_row);
            const float4 q1 = *reinterpret_cast<float4*>(a_row + 4);
            const float4 hcn = sw.g1[slot];   // the entry's conic, staged as (a/2, b, c/2)
            const float4 cn = make_float4(2.f * hcn.x, hcn.y, 2.f * hcn.z, hcn.w);
            // gradients of (mean, mean velocity) and (conic, opacity) record entries: -ddx, -ddy,
            // -ddx t, -ddy t, dsig dx^2 / 2, dsig dx dy, dsig dy^2 / 2, dg G (dsig = -Pn)
            const float4 s0 = make_float4(cn.x * q0.x + cn.y * q0.y, cn.y * q0.x + cn.z * q0.y,
                                          cn.x * q0.z + cn.y * q0.w, cn.y * q0.z + cn.z * q0.w);
            const float4 s1 = make_float4(-0.5f * q1.x, -q1.y, -0.5f * q1.z, q1.w);
            if (s0.x != 0.f || s0.y != 0.f || s0.z != 0.f || s0.w != 0.f || s1.x != 0.f || s1.y != 0.f ||
                s1.z != 0.f || s1.w != 0.f) {
                atomicAdd(gp0 + id, s0);
                atomicAdd(gp1 + id, s1);
            }
            float* df = gr.dfeatures + (int64_t)id * C;
            if ((C & 3) == 0) {
#pragma unroll
                for (int c = 0; c < 16; c += 4) {
                    if (c < C) {
                        const float4 f4 = *reinterpret_cast<float4*>(a_row + 8 + c);
                        if (f4.x != 0.f || f4.y != 0.f || f4.z != 0.f || f4.w != 0.f)
                            atomicAdd(reinterpret_cast<float4*>(df + c), f4);
                    }
                }
            } else {
#pragma unroll
                for (int c = 0; c < 16; c++)
                    if (c < C && a_row[8 + c] != 0.f) atomicAdd(df + c, a_row[8 + c]);
            }
#pragma unroll
            for (int q = 0; q < kRow; q += 4) *reinterpret_cast<float4*>(a_row + q) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
    if (gr.dsensor) {   // one atomic per block (uniform branch)
        __shared__ float s_dt[2];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dtime += __shfl_xor_sync(0xffffffffu, dtime, o);
        if (lane == 0) s_dt[w] = dtime;
        __syncthreads();
        if (threadIdx.x == 0) {
            const float tot = s_dt[0] + s_dt[1];
            if (tot != 0.f) atomicAdd(gr.dsensor + 16 * tc.s + 6, tot);
        }
    }
}

}  // namespace splat
