// head_umma.cu -- training pass of the per-ray lidar decoder (paper Sec. 3.3 decoder, App. B
// loss weights) on the fifth-generation tensor cores.
//
// Training: one CTA per SM, 512 threads, 128-ray tiles: ray q of a tile is TMEM lane q, and the four
// warps w, w + 4, w + 8, w + 12 (the warps that may read lane quarter w) share lanes
// 32 w .. 32 w + 31, each taking 16 of the 64 columns of those rays.  Per tile, in order:
//   Z1 = X W1, Z2 = H1 W2                    M = 128 products into TMEM
//   O = H2 W3, dO (loss derivative), dZ2 = relu'(z2) (dO W3^T)   on the CUDA cores
//   dH1 = dZ2 W2^T;  G2 += dZ2^T [H1 | 1];  G3 += H2^T dO
//   dX = dZ1 W1^T (optional);  G1 += dZ1^T [X | 1]
// The threads wait only for the layer and input-gradient products; the weight-gradient
// products run behind them on their own mbarriers and are waited for when the next tile
// overwrites their operands.
// G1, G2, G3 are M = 64 accumulators over all of the CTA's rays, kept in TMEM and added to
// the FP32 gradient once at the end: G2 = dW2^T with db2 in its last column, G1 = dW1^T
// with db1, G3 = dW3; db3 and the loss are summed on the CUDA cores.
//
// Numerics as the warp-level decoder kernels: weights are exact BF16; activations and
// gradients are FP32 values split into a BF16 high part and a BF16 residual, a product with a
// weight takes two MMAs (high, residual) and a product of two split values three (the
// residual x residual term is below FP32 accumulation noise).  Every activation buffer is
// read by one product as a K-major operand and by a weight-gradient product as an MN-major
// one (umma.cuh): no transposed copies.
#include <cuda_bf16.h>

#include "head_impl.cuh"
#include "status.cuh"
#include "umma.cuh"

namespace splat {

namespace {
constexpr int kTR = 128;                 // rays per tile
constexpr int kXC = 48, kH1C = 80;       // columns of X | 1 and H1 | 1 (padded to 16)
constexpr int kRsX = kXC / 8 * 128, kRsH1 = kH1C / 8 * 128, kRs64 = 64 / 8 * 128, kRsO = 16 / 8 * 128;
constexpr int kRsW = 64 / 8 * 128;       // W1 [32][64] and W2 [64][64]: rows = inputs
constexpr int kRsW3 = 16 / 8 * 128;      // W3 [64][16 (2 used)]
// TMEM columns
constexpr uint32_t kTZ1 = 0, kTZ2 = 64, kTDH1 = 128, kTDX = 192, kTG2 = 256, kTG1 = 336, kTG3 = 384;
constexpr uint32_t kTCols = 512;
constexpr uint32_t kSiteHeadWait = 31;   // status site: an MMA completion wait ran out

constexpr int kThreads = 512;

struct TrainSmem {
    alignas(1024) unsigned char xh[kTR * kXC * 2], xl[kTR * kXC * 2];
    alignas(1024) unsigned char h1h[kTR * kH1C * 2], h1l[kTR * kH1C * 2];
    alignas(1024) unsigned char h2h[kTR * 64 * 2], h2l[kTR * 64 * 2];
    alignas(1024) unsigned char dz2h[kTR * 64 * 2], dz2l[kTR * 64 * 2];
    alignas(1024) unsigned char dz1h[kTR * 64 * 2], dz1l[kTR * 64 * 2];
    alignas(1024) unsigned char doh[kTR * 16 * 2], dol[kTR * 16 * 2];
    alignas(1024) unsigned char w1[32 * 64 * 2], w2[64 * 64 * 2], w3[64 * 16 * 2];
    float w3f[kHHid][kHOut];
    float b1[kHHid], b2[kHHid], b3[kHOut];
    float opart[4][kTR][2];   // per column slice: partial O = H2 W3 of each ray
    float dO[kTR][2];
    uint64_t mb_f;     // the layer and input-gradient products (the critical chain)
    uint64_t mb_g23;   // the weight-gradient products G2, G3 of a tile
    uint64_t mb_g1;    // G1 of a tile
    uint32_t tmem;
};

__device__ __forceinline__ void load_weights(TrainSmem& s, const HeadW& hw) {
    const bf16* w = reinterpret_cast<const bf16*>(hw.w);
    for (int e = threadIdx.x; e < kW1; e += blockDim.x) {
        const int f = e / kHHid, j = e % kHHid;
        *reinterpret_cast<bf16*>(s.w1 + umma::off(f, j, kRsW)) = w[e];
    }
    for (int e = threadIdx.x; e < kW2; e += blockDim.x) {
        const int i = e / kHHid, j = e % kHHid;
        *reinterpret_cast<bf16*>(s.w2 + umma::off(i, j, kRsW)) = w[kW1 + e];
    }
    for (int e = threadIdx.x; e < kHHid * 16; e += blockDim.x) {
        const int i = e / 16, k = e % 16;
        const bf16 v = k < kHOut ? w[kW1 + kW2 + i * kHOut + k] : __float2bfloat16_rn(0.f);
        *reinterpret_cast<bf16*>(s.w3 + umma::off(i, k, kRsW3)) = v;
        if (k < kHOut) s.w3f[i][k] = __bfloat162float(v);
    }
    for (int e = threadIdx.x; e < 2 * kHHid + kHOut; e += blockDim.x) {
        const float v = hw.b[e];
        if (e < kHHid) s.b1[e] = v;
        else if (e < 2 * kHHid) s.b2[e - kHHid] = v;
        else s.b3[e - 2 * kHHid] = v;
    }
}

// Columns [c0, c0 + 8 G) of row `row` into the split planes, two values per conversion.
template <int G>
__device__ __forceinline__ void store_split(unsigned char* hi, unsigned char* lo, int row, int c0, int rs,
                                            const float (&v)[8 * G]) {
#pragma unroll
    for (int g = 0; g < G; g++) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; e++) split_pair(v[8 * g + 2 * e], v[8 * g + 2 * e + 1], h[e], l[e]);
        const int o = umma::off(row, c0 + 8 * g, rs);
        *reinterpret_cast<uint4*>(hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}
}  // namespace

__global__ void __launch_bounds__(kThreads, 1) k_head_train_umma(const float* __restrict__ x, int64_t R, HeadW hw,
                                                                const float* __restrict__ y_int,
                                                                const float* __restrict__ y_drop, float lam_i,
                                                                float lam_d, float* __restrict__ grad, float* loss,
                                                                float* __restrict__ dx) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TrainSmem& s = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, slice = warp >> 2;   // lane quarter and 16-column slice
    const int q = 32 * quarter + lane;                 // this thread's ray (row) of a tile
    const int c16 = 16 * slice;                        // its first of 16 columns
    if (warp == 0) umma::tmem_alloc(&s.tmem, kTCols);
    if (tid == 0) {
        umma::mbar_init(&s.mb_f, 1);
        umma::mbar_init(&s.mb_g23, 1);
        umma::mbar_init(&s.mb_g1, 1);
    }
    load_weights(s, hw);
    if (slice == 0) {   // the constant columns: X | 1 (col 32) and H1 | 1 (col 64), zeros after them
        float c[16];
#pragma unroll
        for (int j = 0; j < 16; j++) c[j] = j == 0 ? 1.f : 0.f;
        store_split<2>(s.xh, s.xl, q, 32, kRsX, c);
        store_split<2>(s.h1h, s.h1l, q, 64, kRsH1, c);
    }
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tm = s.tmem;
    const uint32_t lane_base = tm + ((uint32_t)(32 * quarter) << 16);   // this thread's lane
    const uint32_t ax = umma::smem_addr(s.xh), axl = umma::smem_addr(s.xl);
    const uint32_t ah1 = umma::smem_addr(s.h1h), ah1l = umma::smem_addr(s.h1l);
    const uint32_t ah2 = umma::smem_addr(s.h2h), ah2l = umma::smem_addr(s.h2l);
    const uint32_t adz = umma::smem_addr(s.dz2h), adzl = umma::smem_addr(s.dz2l);
    const uint32_t adz1 = umma::smem_addr(s.dz1h), adz1l = umma::smem_addr(s.dz1l);
    const uint32_t ado = umma::smem_addr(s.doh), adol = umma::smem_addr(s.dol);
    const uint32_t aw1 = umma::smem_addr(s.w1), aw2 = umma::smem_addr(s.w2);
    const float invR = 1.f / (float)R;
    float lsum = 0.f, db3[2] = {0.f, 0.f};
    uint32_t ph_f = 0, ph_g23 = 0, ph_g1 = 0;
    bool first = true, ok = true, bad = false;
    // Waits for the next phase of an mbarrier (each is committed once and waited once per
    // round).  A wait that runs out marks this thread; the next publish() makes the block
    // leave together, so that no thread is left at a barrier.
    auto wait_mb = [&](uint64_t* mb, uint32_t& ph) {
        if (!umma::mbar_wait(mb, ph & 1u)) {
            if (!bad) raise_status(kStatusTimeout, kSiteHeadWait);
            bad = true;
        }
        ph++;
        umma::fence_after_sync();
    };
    // This thread's shared-memory operand writes, for the tensor core; false (on every
    // thread) once any thread's wait has run out.
    auto publish = [&]() -> bool {
        umma::fence_async_smem();
        umma::fence_before_sync();
        const bool any_bad = __syncthreads_or(bad);
        umma::fence_after_sync();
        return !any_bad;
    };
    // the lane quarter's four warps (the threads of the same rays)
    auto quarter_sync = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(1 + quarter) : "memory"); };
    // inputs [8 slice, 8 slice + 8) and labels of this thread's ray of a tile
    auto load_tile = [&](int64_t tile, float (&xv)[8], float& yi, float& yd) {
        const int64_t r = tile * kTR + q;
        if (tile < (R + kTR - 1) / kTR && r < R) {
            const float4* xp = reinterpret_cast<const float4*>(x + r * kHIn + 8 * slice);
            const float4 a = xp[0], b = xp[1];
            xv[0] = a.x; xv[1] = a.y; xv[2] = a.z; xv[3] = a.w;
            xv[4] = b.x; xv[5] = b.y; xv[6] = b.z; xv[7] = b.w;
            yi = slice == 0 ? y_int[r] : 0.f;
            yd = slice == 0 ? y_drop[r] : 0.f;
        } else {
#pragma unroll
            for (int j = 0; j < 8; j++) xv[j] = 0.f;
            yi = yd = 0.f;
        }
    };
    const int64_t tiles = (R + kTR - 1) / kTR;
    float xv[8], yi, yd;
    load_tile(blockIdx.x, xv, yi, yd);
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t r = tile * kTR + q;
        const bool valid = r < R;
        // the previous tile's G1 reads X and dZ1
        if (!first) wait_mb(&s.mb_g1, ph_g1);
        store_split<1>(s.xh, s.xl, q, 8 * slice, kRsX, xv);
        const float y_i = yi, y_d = yd;
        load_tile(tile + gridDim.x, xv, yi, yd);   // the next tile's, in flight meanwhile
        if (!(ok = publish())) break;
        // Z1 = X W1
        if (tid == 0) {
            constexpr uint32_t id = umma::idesc_bf16(128, 64, false, true);
#pragma unroll
            for (int ks = 0; ks < 2; ks++) {
                const uint64_t b = umma::desc_mn(aw1, kRsW, ks);
                umma::mma(tm + kTZ1, umma::desc_k(ax, kRsX, ks), b, id, ks > 0);
                umma::mma(tm + kTZ1, umma::desc_k(axl, kRsX, ks), b, id, true);
            }
            umma::commit(&s.mb_f);
        }
        wait_mb(&s.mb_f, ph_f);
        uint32_t m1 = 0u, m2 = 0u;   // ReLU masks of this thread's 16 columns
        {
            float v[16];
            umma::tmem_ld16(lane_base + kTZ1 + c16, v);
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const float z = v[j] + s.b1[c16 + j];
                v[j] = fmaxf(z, 0.f);
                if (z > 0.f) m1 |= 1u << j;
            }
            // the previous tile's G2 and G3 read H1, H2, dZ2 and dO
            if (!first) wait_mb(&s.mb_g23, ph_g23);
            store_split<2>(s.h1h, s.h1l, q, c16, kRsH1, v);
        }
        if (!(ok = publish())) break;
        // Z2 = H1 W2
        if (tid == 0) {
            constexpr uint32_t id = umma::idesc_bf16(128, 64, false, true);
#pragma unroll
            for (int ks = 0; ks < 4; ks++) {
                const uint64_t b = umma::desc_mn(aw2, kRsW, ks);
                umma::mma(tm + kTZ2, umma::desc_k(ah1, kRsH1, ks), b, id, ks > 0);
                umma::mma(tm + kTZ2, umma::desc_k(ah1l, kRsH1, ks), b, id, true);
            }
            umma::commit(&s.mb_f);
        }
        wait_mb(&s.mb_f, ph_f);
        float h2[16];
        {
            umma::tmem_ld16(lane_base + kTZ2 + c16, h2);
            float o0 = 0.f, o1 = 0.f;   // this slice's part of O = H2 W3 (FP32, CUDA cores)
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const float z = h2[j] + s.b2[c16 + j];
                h2[j] = fmaxf(z, 0.f);
                if (z > 0.f) m2 |= 1u << j;
                o0 = fmaf(h2[j], s.w3f[c16 + j][0], o0);
                o1 = fmaf(h2[j], s.w3f[c16 + j][1], o1);
            }
            s.opart[slice][q][0] = o0;
            s.opart[slice][q][1] = o1;
            store_split<2>(s.h2h, s.h2l, q, c16, kRs64, h2);
        }
        quarter_sync();
        if (slice == 0) {   // the ray's outputs, loss and dL/dO
            const float o0 = s.b3[0] + ((s.opart[0][q][0] + s.opart[1][q][0]) + (s.opart[2][q][0] + s.opart[3][q][0]));
            const float o1 = s.b3[1] + ((s.opart[0][q][1] + s.opart[1][q][1]) + (s.opart[2][q][1] + s.opart[3][q][1]));
            float dO0 = 0.f, dO1 = 0.f;
            if (valid) {
                const float sg = 1.f / (1.f + __expf(-o0));
                const float e = sg - y_i;
                const float bce = fmaxf(o1, 0.f) - o1 * y_d + log1pf(__expf(-fabsf(o1)));
                lsum += lam_i * e * e * invR + lam_d * bce * invR;
                dO0 = lam_i * 2.f * e * sg * (1.f - sg) * invR;
                dO1 = lam_d * (1.f / (1.f + __expf(-o1)) - y_d) * invR;
            }
            db3[0] += dO0;
            db3[1] += dO1;
            s.dO[q][0] = dO0;
            s.dO[q][1] = dO1;
            float dov[16];
#pragma unroll
            for (int j = 0; j < 16; j++) dov[j] = 0.f;
            dov[0] = dO0;
            dov[1] = dO1;
            store_split<2>(s.doh, s.dol, q, 0, kRsO, dov);
        }
        quarter_sync();
        {   // dZ2 = relu'(z2) (dO W3^T)
            const float dO0 = s.dO[q][0], dO1 = s.dO[q][1];
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const float d = dO0 * s.w3f[c16 + j][0] + dO1 * s.w3f[c16 + j][1];
                v[j] = ((m2 >> j) & 1u) ? d : 0.f;
            }
            store_split<2>(s.dz2h, s.dz2l, q, c16, kRs64, v);
        }
        if (!(ok = publish())) break;
        // dH1 = dZ2 W2^T (waited for); then G2 += dZ2^T [H1 | 1] and G3 += H2^T dO (not)
        if (tid == 0) {
            {
                constexpr uint32_t id = umma::idesc_bf16(128, 64, false, false);
#pragma unroll
                for (int ks = 0; ks < 4; ks++) {
                    const uint64_t b = umma::desc_k(aw2, kRsW, ks);
                    umma::mma(tm + kTDH1, umma::desc_k(adz, kRs64, ks), b, id, ks > 0);
                    umma::mma(tm + kTDH1, umma::desc_k(adzl, kRs64, ks), b, id, true);
                }
            }
            umma::commit(&s.mb_f);
            constexpr uint32_t id2 = umma::idesc_bf16(64, kH1C, true, true);
            constexpr uint32_t id3 = umma::idesc_bf16(64, 16, true, true);
            const uint64_t ah0 = umma::desc_mn(adz, kRs64, 0), al0 = umma::desc_mn(adzl, kRs64, 0);
            const uint64_t bh0 = umma::desc_mn(ah1, kRsH1, 0), bl0 = umma::desc_mn(ah1l, kRsH1, 0);
            const uint64_t ch0 = umma::desc_mn(ah2, kRs64, 0), cl0 = umma::desc_mn(ah2l, kRs64, 0);
            const uint64_t dh0 = umma::desc_mn(ado, kRsO, 0), dl0 = umma::desc_mn(adol, kRsO, 0);
#pragma unroll
            for (int ks = 0; ks < kTR / 16; ks++) {
                const uint64_t ah = umma::step_mn(ah0, kRs64, ks), al = umma::step_mn(al0, kRs64, ks);
                const uint64_t bh = umma::step_mn(bh0, kRsH1, ks), bl = umma::step_mn(bl0, kRsH1, ks);
                umma::mma(tm + kTG2, ah, bh, id2, !(first && ks == 0));
                umma::mma(tm + kTG2, ah, bl, id2, true);
                umma::mma(tm + kTG2, al, bh, id2, true);
                const uint64_t ch = umma::step_mn(ch0, kRs64, ks), cl = umma::step_mn(cl0, kRs64, ks);
                const uint64_t dh = umma::step_mn(dh0, kRsO, ks), dl = umma::step_mn(dl0, kRsO, ks);
                umma::mma(tm + kTG3, ch, dh, id3, !(first && ks == 0));
                umma::mma(tm + kTG3, ch, dl, id3, true);
                umma::mma(tm + kTG3, cl, dh, id3, true);
            }
            umma::commit(&s.mb_g23);
        }
        wait_mb(&s.mb_f, ph_f);
        {   // dZ1 = relu'(z1) dH1
            float v[16];
            umma::tmem_ld16(lane_base + kTDH1 + c16, v);
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] = ((m1 >> j) & 1u) ? v[j] : 0.f;
            store_split<2>(s.dz1h, s.dz1l, q, c16, kRs64, v);
        }
        if (!(ok = publish())) break;
        // dX = dZ1 W1^T (optional, waited for); G1 += dZ1^T [X | 1] (not)
        if (tid == 0) {
            if (dx) {
                constexpr uint32_t id = umma::idesc_bf16(128, 32, false, false);
#pragma unroll
                for (int ks = 0; ks < 4; ks++) {
                    const uint64_t b = umma::desc_k(aw1, kRsW, ks);
                    umma::mma(tm + kTDX, umma::desc_k(adz1, kRs64, ks), b, id, ks > 0);
                    umma::mma(tm + kTDX, umma::desc_k(adz1l, kRs64, ks), b, id, true);
                }
                umma::commit(&s.mb_f);
            }
            constexpr uint32_t id1 = umma::idesc_bf16(64, kXC, true, true);
            const uint64_t ah0 = umma::desc_mn(adz1, kRs64, 0), al0 = umma::desc_mn(adz1l, kRs64, 0);
            const uint64_t bh0 = umma::desc_mn(ax, kRsX, 0), bl0 = umma::desc_mn(axl, kRsX, 0);
#pragma unroll
            for (int ks = 0; ks < kTR / 16; ks++) {
                const uint64_t ah = umma::step_mn(ah0, kRs64, ks), al = umma::step_mn(al0, kRs64, ks);
                const uint64_t bh = umma::step_mn(bh0, kRsX, ks), bl = umma::step_mn(bl0, kRsX, ks);
                umma::mma(tm + kTG1, ah, bh, id1, !(first && ks == 0));
                umma::mma(tm + kTG1, ah, bl, id1, true);
                umma::mma(tm + kTG1, al, bh, id1, true);
            }
            umma::commit(&s.mb_g1);
        }
        first = false;
        if (dx) {   // columns [8 slice, 8 slice + 8) of dX (the loads are warp-collective)
            wait_mb(&s.mb_f, ph_f);
            float v[16], w[8];
            umma::tmem_ld16(lane_base + kTDX + 16 * (slice >> 1), v);   // columns 16 (slice / 2) ..
#pragma unroll
            for (int e = 0; e < 8; e++) w[e] = (slice & 1) ? v[8 + e] : v[e];   // this slice's half
            if (valid) {
                float4* dp = reinterpret_cast<float4*>(dx + r * kHIn + 8 * slice);
                dp[0] = make_float4(w[0], w[1], w[2], w[3]);
                dp[1] = make_float4(w[4], w[5], w[6], w[7]);
            }
        }
    }
    // the last tile's weight-gradient products
    if (ok && !first) {
        wait_mb(&s.mb_g23, ph_g23);
        wait_mb(&s.mb_g1, ph_g1);
        ok = publish();
    }
    // flush: M = 64 rows sit in the first 16 lanes of each lane quarter; W1 b1 W2 b2 W3 b3
    if (ok && !first) {
        float* gW1 = grad;
        float* gb1 = grad + kW1;
        float* gW2 = gb1 + kHHid;
        float* gb2 = gW2 + kW2;
        float* gW3 = gb2 + kHHid;
        const int j = 16 * quarter + lane;   // unit of this lane (lanes 0..15)
        // G2: 80 columns in five 16-column groups (slices 0..3, and slice 0 the fifth);
        // G1: 48 columns (slices 0..2); G3: 16 columns (slice 3)
        for (int grp = slice; grp < 5; grp += 4) {
            float v[16];
            umma::tmem_ld16(lane_base + kTG2 + 16 * grp, v);
            if (lane < 16) {
#pragma unroll
                for (int c = 0; c < 16; c++) {
                    const int n = 16 * grp + c;
                    if (n < kHHid) atomicAdd(gW2 + n * kHHid + j, v[c]);
                    else if (n == kHHid) atomicAdd(gb2 + j, v[c]);
                }
            }
        }
        if (slice < 3) {
            float v[16];
            umma::tmem_ld16(lane_base + kTG1 + 16 * slice, v);
            if (lane < 16) {
#pragma unroll
                for (int c = 0; c < 16; c++) {
                    const int n = 16 * slice + c;
                    if (n < kHIn) atomicAdd(gW1 + n * kHHid + j, v[c]);
                    else if (n == kHIn) atomicAdd(gb1 + j, v[c]);
                }
            }
        } else {
            float v[16];
            umma::tmem_ld16(lane_base + kTG3, v);
            if (lane < 16) {
                atomicAdd(gW3 + j * kHOut, v[0]);
                atomicAdd(gW3 + j * kHOut + 1, v[1]);
            }
        }
        if (slice == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
                db3[0] += __shfl_xor_sync(0xffffffffu, db3[0], o);
                db3[1] += __shfl_xor_sync(0xffffffffu, db3[1], o);
            }
            if (lane == 0) {
                if (loss) atomicAdd(loss, lsum);
                atomicAdd(gW3 + kW3, db3[0]);
                atomicAdd(gW3 + kW3 + 1, db3[1]);
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_free(tm, kTCols);
}

void launch_head_train_umma(const float* x, int64_t R, const HeadW& hw, const float* y_int, const float* y_drop,
                            float lam_i, float lam_d, float* grad, float* loss, float* dx, cudaStream_t st) {
    if (R <= 0) return;
    const size_t sm = sizeof(TrainSmem);
    cudaFuncSetAttribute(k_head_train_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t blocks = (R + kTR - 1) / kTR;
    if (blocks > sms) blocks = sms;   // one CTA per SM: its Tensor Memory columns are all of the SM's
    k_head_train_umma<<<(unsigned)blocks, kThreads, sm, st>>>(x, R, hw, y_int, y_drop, lam_i, lam_d, grad, loss, dx);
}

}  // namespace splat
