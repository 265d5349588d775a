// head.cu -- the per-ray lidar decoder: rendered features + ray direction -> 64 -> 64 -> 2
// (intensity logit, ray-drop logit).  Paper Sec. 3.3 (features concatenated with the ray
// direction, decoded by a small MLP to intensity and ray-drop probability), App. B (a
// lightweight two-hidden-layer MLP; loss weights lambda_intens = 1, lambda_raydrop = 0.1
// in Eq. loss_fn).
//
// Weights are stored in BF16 (W1 | W2 | W3 packed, row-major [in][out]) with FP32 biases
// and FP32 master copies for the optimiser.  Activations and gradients stay FP32 values:
// each is split into a BF16 high part and a BF16 residual, and a product with an exact
// BF16 weight takes two MMAs (high and residual), a product of two split values three (the
// residual x residual term is below FP32 accumulation noise), so the decoder's numerics
// are those of FP32 activations with BF16 weights.
//
// This file holds the forward (inference, and the decoder fused into the lidar raster's
// epilogue) on warp-level MMAs (mma.sync m16n8k16): a warp owns 16 rays (one MMA row tile)
// and a layer's accumulator fragments (rows = rays, columns = units) are exactly the next
// layer's A-operand fragments, so activations pass from layer to layer in registers.  The
// training pass runs on the fifth-generation tensor cores (head_umma.cu).
#include <cuda_bf16.h>

#include "head_impl.cuh"
#include "raster_impl.cuh"

namespace splat {
__global__ void __launch_bounds__(kHeadThreads) k_head_fwd(const float* __restrict__ x, int64_t R, HeadW hw,
                                                           float* __restrict__ out) {
    __shared__ HeadSmemW s;
    load_head_weights(s, hw);
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t tiles = (R + 15) / 16;
    const int64_t stride = (int64_t)gridDim.x * kHeadWarps;
    int64_t tile = (int64_t)blockIdx.x * kHeadWarps + (threadIdx.x >> 5);
    float2 cur[2][4];
    if (tile < tiles) load_x_raw(x, tile * 16, R, cur);
    for (; tile < tiles; tile += stride) {
        const int64_t r0 = tile * 16;
        float2 nxt[2][4];   // the next tile's inputs are in flight during this tile's MMAs
        if (tile + stride < tiles) load_x_raw(x, (tile + stride) * 16, R, nxt);
        SplitA xa[2];
#pragma unroll
        for (int ks = 0; ks < 2; ks++)
#pragma unroll
            for (int q = 0; q < 4; q++) split_pair(cur[ks][q].x, cur[ks][q].y, xa[ks].h[q], xa[ks].l[q]);
        HeadFwd f;
        head_forward_tile(s, xa, f);
#pragma unroll
        for (int ks = 0; ks < 2; ks++)
#pragma unroll
            for (int q = 0; q < 4; q++) cur[ks][q] = nxt[ks][q];
        if (t == 0) {
            if (r0 + g < R) reinterpret_cast<float2*>(out)[r0 + g] = make_float2(f.o[0], f.o[1]);
            if (r0 + g + 8 < R) reinterpret_cast<float2*>(out)[r0 + g + 8] = make_float2(f.o[2], f.o[3]);
        }
    }
}

// Per-iteration shared buffers of a training block (64 rays): transposed BF16 split copies
// of X, H1, dZ1, dZ2 for the weight-gradient contractions; H2 and dO in FP32.
// Adam on the FP32 masters (W1 b1 W2 b2 W3 b3), then the BF16 weight copy and FP32 biases
// the decoder reads.
__global__ void k_head_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float beta1, float beta2, float eps, float c1,
                            float c2, uint16_t* __restrict__ wbf, float* __restrict__ bias) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = beta1 * m[i] + (1.f - beta1) * gi;
        const float vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        // packed index: W1 [0, kW1), b1, W2, b2, W3, b3
        int64_t k = i;
        if (k < kW1) { wbf[k] = __bfloat16_as_ushort(__float2bfloat16_rn(pi)); continue; }
        k -= kW1;
        if (k < kHHid) { bias[k] = pi; continue; }
        k -= kHHid;
        if (k < kW2) { wbf[kW1 + k] = __bfloat16_as_ushort(__float2bfloat16_rn(pi)); continue; }
        k -= kW2;
        if (k < kHHid) { bias[kHHid + k] = pi; continue; }
        k -= kHHid;
        if (k < kW3) { wbf[kW1 + kW2 + k] = __bfloat16_as_ushort(__float2bfloat16_rn(pi)); continue; }
        k -= kW3;
        bias[2 * kHHid + k] = pi;
    }
}

// x[r] = [features of ray r (C values), unit direction (cos w cos p, cos w sin p, sin w)]
__global__ void k_head_inputs(const __grid_constant__ SensorDev S, const float* __restrict__ feat, int C,
                              float* __restrict__ x) {
    const int64_t R = (int64_t)S.nb * S.naz;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(r / S.naz), a = (int)(r - (int64_t)b * S.naz);
        float phi, om;
        if (S.rays) {
            phi = S.rays[3 * r];
            om = S.rays[3 * r + 1];
        } else {
            phi = (a + 0.5f) * S.az_res;
            om = S.elev[b];
        }
        float* xr = x + r * kHIn;
        for (int c = 0; c < C; c++) xr[c] = feat[r * C + c];
        float sp, cp, sw, cw;
        sincosf(phi, &sp, &cp);
        sincosf(om, &sw, &cw);
        xr[C] = cw * cp;
        xr[C + 1] = cw * sp;
        xr[C + 2] = sw;
    }
}

// ---------------------------------------------------------------------------------
// Lidar forward with the decoder in its epilogue (Sec. 3.3: each ray's rendered features
// and its direction decoded into intensity and ray-drop logits).  The block renders its
// lidar tile exactly as k_raster_fwd does (same traversal, same outputs), then reuses
// its staging memory for the decoder's forward weights and the tile's 256 input rows
// [29 features, unit direction]; each warp decodes its 32 rays as two 16-ray tensor-core
// tiles (head_forward_tile, the unfused decoder's arithmetic).  The features never
// travel through HBM to reach the decoder.
// ---------------------------------------------------------------------------------
constexpr int kXRow = 40;   // floats per input row in shared memory (conflict-free fragment loads)

template <int TW, int TH>
struct FusedHeadSmem {
    static constexpr int NT = TW * TH;
    static constexpr size_t head = (sizeof(HeadSmemFwd) + 15) & ~size_t(15);
    static constexpr size_t bytes_head = head + sizeof(float) * NT * kXRow;
    static constexpr size_t bytes_stage = sizeof(Stage<32, NT, true>);
    static constexpr size_t bytes = bytes_head > bytes_stage ? bytes_head : bytes_stage;
};

template <int TW, int TH>
__global__ void __launch_bounds__(TW* TH) k_lidar_fwd_head(const __grid_constant__ Frame fr, RasterIn in,
                                                           RasterOut out, HeadW hw, float* __restrict__ head_out) {
    constexpr int CM = 32, NT = TW * TH;
    static_assert(RaysPerThread<CM, false, true, NT>::value == 1 && NT % 32 == 0, "one ray per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Stage<CM, NT, true>& sm = *reinterpret_cast<Stage<CM, NT, true>*>(smem_raw);
    TileCtx tc;
    RayCtx r[1];
    block_setup<TW, TH, true, false, 1, NT>(fr, in, tc, r);
    const int2 range = load_range(in, tc.gtile);
    const TileBox box{};
    float2 F[1][CM / 2];
#pragma unroll
    for (int c = 0; c < CM / 2; c++) F[0][c] = make_float2(0.f, 0.f);
    FwdState st[1];
    forward_tile<CM, TW, TH, true, 1, true, false>(sm, in, tc, box, r, range, st, F);
    const int C = in.C;   // kHIn - 3
    if (r[0].inside) {
        const int64_t o = r[0].o;
        if (out.feat) {
            float* fo = out.feat + o * C;
#pragma unroll
            for (int c = 0; c < CM; c++)
                if (c < C) fo[c] = (c & 1) ? F[0][c / 2].y : F[0][c / 2].x;
        }
        if (out.T) out.T[o] = st[0].T;
        if (out.last) out.last[o] = st[0].last;
        out.range_exp[o] = st[0].de;
        if (out.range_med) out.range_med[o] = st[0].dm;
        out.alpha[o] = 1.f - st[0].T;
    }
    __syncthreads();   // the staging memory is free: decoder weights and input rows
    HeadSmemFwd& hs = *reinterpret_cast<HeadSmemFwd*>(smem_raw);
    float* xs = reinterpret_cast<float*>(smem_raw + FusedHeadSmem<TW, TH>::head);
    load_head_fwd_weights(hs, hw);
    {
        float* xr = xs + threadIdx.x * kXRow;
#pragma unroll
        for (int c = 0; c < CM; c++)
            if (c < C) xr[c] = (c & 1) ? F[0][c / 2].y : F[0][c / 2].x;
        // the unit ray direction, as splat_head_inputs forms it
        float sp, cp, sw, cw;
        sincosf(r[0].pa, &sp, &cp);
        sincosf(r[0].pb, &sw, &cw);
        xr[C] = cw * cp;
        xr[C + 1] = cw * sp;
        xr[C + 2] = sw;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int half = 0; half < 2; half++) {
        const int row0 = 32 * warp + 16 * half;   // the tile's rays are threads row0 .. row0 + 15
        SplitA xa[2];
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int row = row0 + g + ((q & 1) ? 8 : 0);
                const int col = 16 * ks + ((q & 2) ? 8 : 0) + 2 * t;
                const float2 v = *reinterpret_cast<const float2*>(xs + row * kXRow + col);
                split_pair(v.x, v.y, xa[ks].h[q], xa[ks].l[q]);
            }
        }
        HeadFwd f;
        head_forward_tile(hs, xa, f);
        // rows g and g + 8 of the tile belong to lanes 16 half + g (+ 8) of this warp
        const int64_t oa = __shfl_sync(0xffffffffu, r[0].o, 16 * half + g);
        const int64_t ob = __shfl_sync(0xffffffffu, r[0].o, 16 * half + g + 8);
        const bool ia = __shfl_sync(0xffffffffu, (int)r[0].inside, 16 * half + g);
        const bool ib = __shfl_sync(0xffffffffu, (int)r[0].inside, 16 * half + g + 8);
        if (t == 0) {
            if (ia) reinterpret_cast<float2*>(head_out)[oa] = make_float2(f.o[0], f.o[1]);
            if (ib) reinterpret_cast<float2*>(head_out)[ob] = make_float2(f.o[2], f.o[3]);
        }
    }
}

bool launch_lidar_fwd_head(int tw, int th, const Frame& fr, int blocks, const RasterIn& in, const RasterOut& out,
                           const HeadW& hw, float* head_out, cudaStream_t st) {
    if (tw != 32 || th != 8 || in.C != kHIn - 3) return false;
    constexpr size_t sm = FusedHeadSmem<32, 8>::bytes;
    auto k = k_lidar_fwd_head<32, 8>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (blocks > 0) k<<<blocks, 256, sm, st>>>(fr, in, out, hw, head_out);
    return true;
}


void launch_head_fwd(const float* x, int64_t R, const HeadW& hw, float* out, cudaStream_t st) {
    if (R <= 0) return;
    int64_t blocks = ((R + 15) / 16 + kHeadWarps - 1) / kHeadWarps;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_head_fwd<<<(unsigned)blocks, kHeadThreads, 0, st>>>(x, R, hw, out);
}

void launch_head_train_umma(const float* x, int64_t R, const HeadW& hw, const float* y_int, const float* y_drop,
                            float lam_i, float lam_d, float* grad, float* loss, float* dx, cudaStream_t st);

void launch_head_train(const float* x, int64_t R, const HeadW& hw, const float* y_int, const float* y_drop, float lam_i,
                       float lam_d, float* grad, float* loss, float* dx, cudaStream_t st) {
    launch_head_train_umma(x, R, hw, y_int, y_drop, lam_i, lam_d, grad, loss, dx, st);
}

void launch_head_adam(float* p, const float* g, float* m, float* v, float lr, float beta1, float beta2, float eps,
                      int64_t step, uint16_t* wbf, float* bias, cudaStream_t st) {
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_head_adam<<<(kHeadParams + 255) / 256, 256, 0, st>>>(p, g, m, v, kHeadParams, lr, beta1, beta2, eps, c1, c2,
                                                          wbf, bias);
}

void launch_head_inputs(const SensorDev& S, const float* feat, int C, float* x, cudaStream_t st) {
    const int64_t R = (int64_t)S.nb * S.naz;
    if (R <= 0) return;
    int64_t blocks = (R + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_head_inputs<<<(unsigned)blocks, 256, 0, st>>>(S, feat, C, x);
}

int head_param_count() { return kHeadParams; }

}  // namespace splat
