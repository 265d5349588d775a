// head.cu -- the per-ray lidar decoder: rendered features + ray direction -> 64 -> 64 -> 2
// (intensity logit, ray-drop logit).  Paper Sec. 3.3 (features concatenated with the ray
// direction, decoded by a small MLP to intensity and ray-drop probability), App. B (a
// lightweight two-hidden-layer MLP; loss weights lambda_intens = 1, lambda_raydrop = 0.1
// in Eq. loss_fn).
//
// Weights are stored in BF16 (W1 | W2 | W3 packed, row-major [in][out]) with FP32 biases
// and FP32 master copies for the optimiser.  Every contraction runs on the tensor cores
// (mma.sync m16n8k16, BF16 operands, FP32 accumulation).  Activations and gradients stay
// FP32 values: each is split into a BF16 high part and a BF16 residual, and a product
// with an exact BF16 weight takes two MMAs (high and residual), a product of two split
// values three (the residual x residual term is below FP32 accumulation noise), so the
// decoder's numerics are those of FP32 activations with BF16 weights.
//
// A warp owns 16 rays (one MMA row tile).  A layer's accumulator fragments (rows = rays,
// columns = units) are exactly the next layer's A-operand fragments, so activations pass
// from layer to layer in registers.  Training blocks take 64 rays (4 warps) at a time:
// after each warp's forward and backward, the weight gradients dW = A^T dZ contract over
// the block's rays from transposed BF16 copies in shared memory, and stay in registers
// across a persistent grid until one flush per block.
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
struct HeadTrainSmem {
    HeadSmemW w;
    bf16 xt_h[kHIn][kPR], xt_l[kHIn][kPR];
    bf16 h1t_h[kHHid][kPR], h1t_l[kHHid][kPR];
    bf16 z1t_h[kHHid][kPR], z1t_l[kHHid][kPR];
    bf16 z2t_h[kHHid][kPR], z2t_l[kHHid][kPR];
    float h2[kHeadRays][kHHid];
    float dO[kHeadRays][kHOut];
};

// Transposed split store of one C tile: values of rows (rays) g and g + 8, columns
// (units) c0 and c0 + 1.
__device__ __forceinline__ void store_t(bf16 (*th)[kPR], bf16 (*tl)[kPR], const float (&d)[4], int c0, int ray) {
    bf16 h, l;
    split_one(d[0], h, l);
    th[c0][ray] = h;
    tl[c0][ray] = l;
    split_one(d[1], h, l);
    th[c0 + 1][ray] = h;
    tl[c0 + 1][ray] = l;
    split_one(d[2], h, l);
    th[c0][ray + 8] = h;
    tl[c0][ray + 8] = l;
    split_one(d[3], h, l);
    th[c0 + 1][ray + 8] = h;
    tl[c0 + 1][ray + 8] = l;
}

// A fragment (rows = units r0.., k = rays k0..) and B fragment (k = rays k0.., n = units
// n0..) of the weight-gradient products, from transposed [unit][ray] copies.
__device__ __forceinline__ void ld_at(const bf16 (*tt)[kPR], int r0, int k0, uint32_t (&a)[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    a[0] = ld2(&tt[r0 + g][k0 + 2 * t]);
    a[1] = ld2(&tt[r0 + g + 8][k0 + 2 * t]);
    a[2] = ld2(&tt[r0 + g][k0 + 8 + 2 * t]);
    a[3] = ld2(&tt[r0 + g + 8][k0 + 8 + 2 * t]);
}

// Loss lam_i mean (sigmoid(o0) - y_int)^2 + lam_d mean BCE(o1, y_drop) over R rays; adds
// its gradients to grad (W1 b1 W2 b2 W3 b3, FP32) and, if dx is given, writes dL/dx.
__global__ void __launch_bounds__(kHeadThreads) k_head_train(const float* __restrict__ x, int64_t R, HeadW hw,
                                                            const float* __restrict__ y_int,
                                                            const float* __restrict__ y_drop, float lam_i,
                                                            float lam_d, float* __restrict__ grad, float* loss,
                                                            float* __restrict__ dx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HeadTrainSmem& s = *reinterpret_cast<HeadTrainSmem*>(smem_raw);
    load_head_weights(s.w, hw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
    // persistent accumulators: dW2 row tile `warp` (8 n-tiles), dW1 row tile warp & 1 with
    // n-tiles 4 (warp >> 1) .. + 3, and one CUDA-core output each of dW3 / biases
    float aw2[8][4], aw1[4][4];
#pragma unroll
    for (int j = 0; j < 8; j++)
#pragma unroll
        for (int e = 0; e < 4; e++) aw2[j][e] = 0.f;
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int e = 0; e < 4; e++) aw1[j][e] = 0.f;
    float aw3 = 0.f, ab = 0.f, ab3 = 0.f, lsum = 0.f;
    const float invR = 1.f / (float)R;
    const int64_t iters = (R + kHeadRays - 1) / kHeadRays;
    const int ray = 16 * warp + g;   // this lane's rows within the block's 64 rays: ray, ray + 8
    for (int64_t it = blockIdx.x; it < iters; it += gridDim.x) {
        const int64_t r0 = it * kHeadRays + 16 * warp;
        __syncthreads();   // weights loaded / previous iteration's contractions done
        SplitA xa[2];
        float xv[2][4][2];
        load_x_frags(x, r0, R, xa, xv);
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int col = 16 * ks + ((q & 2) ? 8 : 0) + 2 * t, rr = ray + ((q & 1) ? 8 : 0);
                bf16 h, l;
                split_one(xv[ks][q][0], h, l);
                s.xt_h[col][rr] = h;
                s.xt_l[col][rr] = l;
                split_one(xv[ks][q][1], h, l);
                s.xt_h[col + 1][rr] = h;
                s.xt_l[col + 1][rr] = l;
            }
        }
        HeadFwd f;
        head_forward_tile(s.w, xa, f);
        // H1 (transposed, for dW2) and H2 (FP32, for dW3) from the fragments
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const int ks = nt >> 1, q = (nt & 1) * 2;
            float d[4];
            {
                const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&f.h1[ks].h[q]));
                const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&f.h1[ks].l[q]));
                const float2 c = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&f.h1[ks].h[q + 1]));
                const float2 e = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&f.h1[ks].l[q + 1]));
                d[0] = a.x + b.x;
                d[1] = a.y + b.y;
                d[2] = c.x + e.x;
                d[3] = c.y + e.y;
            }
            store_t(s.h1t_h, s.h1t_l, d, 8 * nt + 2 * t, ray);
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&f.h2[ks].h[q]));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&f.h2[ks].l[q]));
            const float2 c = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&f.h2[ks].h[q + 1]));
            const float2 e = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&f.h2[ks].l[q + 1]));
            s.h2[ray][8 * nt + 2 * t] = a.x + b.x;
            s.h2[ray][8 * nt + 2 * t + 1] = a.y + b.y;
            s.h2[ray + 8][8 * nt + 2 * t] = c.x + e.x;
            s.h2[ray + 8][8 * nt + 2 * t + 1] = c.y + e.y;
        }
        // loss and dL/dO on the lanes holding the outputs (t == 0), rows g and g + 8
        float dO[4] = {0.f, 0.f, 0.f, 0.f};
        if (t == 0) {
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int64_t r = r0 + g + 8 * h;
                if (r < R) {
                    const float o0 = f.o[2 * h], o1 = f.o[2 * h + 1];
                    const float sg = 1.f / (1.f + __expf(-o0));
                    const float e = sg - y_int[r];
                    const float y = y_drop[r];
                    const float bce = fmaxf(o1, 0.f) - o1 * y + log1pf(__expf(-fabsf(o1)));
                    lsum += lam_i * e * e * invR + lam_d * bce * invR;
                    dO[2 * h] = lam_i * 2.f * e * sg * (1.f - sg) * invR;
                    dO[2 * h + 1] = lam_d * (1.f / (1.f + __expf(-o1)) - y) * invR;
                }
            }
            s.dO[ray][0] = dO[0];
            s.dO[ray][1] = dO[1];
            s.dO[ray + 8][0] = dO[2];
            s.dO[ray + 8][1] = dO[3];
        }
#pragma unroll
        for (int e = 0; e < 4; e++) dO[e] = __shfl_sync(0xffffffffu, dO[e], lane & ~3);
        // dZ2 = relu'(z2) (dO W3^T), as fragments and transposed
        SplitA z2[4];
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            const int j = 8 * nt + 2 * t;
            float d[4];
            d[0] = dO[0] * s.w.w3[j][0] + dO[1] * s.w.w3[j][1];
            d[1] = dO[0] * s.w.w3[j + 1][0] + dO[1] * s.w.w3[j + 1][1];
            d[2] = dO[2] * s.w.w3[j][0] + dO[3] * s.w.w3[j][1];
            d[3] = dO[2] * s.w.w3[j + 1][0] + dO[3] * s.w.w3[j + 1][1];
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (!((f.m2 >> (4 * nt + e)) & 1u)) d[e] = 0.f;
            c_to_a(d, nt, z2);
            store_t(s.z2t_h, s.z2t_l, d, j, ray);
        }
        // dZ1 = relu'(z1) (dZ2 W2^T)
        SplitA z1[4];
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 4; ks++) {
                const uint32_t b0 = ld2(&s.w.w2[8 * nt + g][16 * ks + 2 * t]);
                const uint32_t b1 = ld2(&s.w.w2[8 * nt + g][16 * ks + 8 + 2 * t]);
                mma16816(d, z2[ks].h, b0, b1);
                mma16816(d, z2[ks].l, b0, b1);
            }
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (!((f.m1 >> (4 * nt + e)) & 1u)) d[e] = 0.f;
            c_to_a(d, nt, z1);
            store_t(s.z1t_h, s.z1t_l, d, 8 * nt + 2 * t, ray);
        }
        if (dx) {   // dX = dZ1 W1^T
#pragma unroll
            for (int nt = 0; nt < 4; nt++) {
                float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int ks = 0; ks < 4; ks++) {
                    const uint32_t b0 = ld2(&s.w.w1[8 * nt + g][16 * ks + 2 * t]);
                    const uint32_t b1 = ld2(&s.w.w1[8 * nt + g][16 * ks + 8 + 2 * t]);
                    mma16816(d, z1[ks].h, b0, b1);
                    mma16816(d, z1[ks].l, b0, b1);
                }
                const int col = 8 * nt + 2 * t;
                if (r0 + g < R) *reinterpret_cast<float2*>(dx + (r0 + g) * kHIn + col) = make_float2(d[0], d[1]);
                if (r0 + g + 8 < R)
                    *reinterpret_cast<float2*>(dx + (r0 + g + 8) * kHIn + col) = make_float2(d[2], d[3]);
            }
        }
        __syncthreads();   // the block's transposed copies are complete
        // dW2 += H1^T dZ2 (rows 16 warp .., all 64 columns), K = the block's 64 rays
#pragma unroll
        for (int ks = 0; ks < kHeadRays / 16; ks++) {
            uint32_t ah[4], al[4];
            ld_at(s.h1t_h, 16 * warp, 16 * ks, ah);
            ld_at(s.h1t_l, 16 * warp, 16 * ks, al);
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                const uint32_t bh0 = ld2(&s.z2t_h[8 * nt + g][16 * ks + 2 * t]);
                const uint32_t bh1 = ld2(&s.z2t_h[8 * nt + g][16 * ks + 8 + 2 * t]);
                const uint32_t bl0 = ld2(&s.z2t_l[8 * nt + g][16 * ks + 2 * t]);
                const uint32_t bl1 = ld2(&s.z2t_l[8 * nt + g][16 * ks + 8 + 2 * t]);
                mma16816(aw2[nt], ah, bh0, bh1);
                mma16816(aw2[nt], ah, bl0, bl1);
                mma16816(aw2[nt], al, bh0, bh1);
            }
        }
        // dW1 += X^T dZ1 (rows 16 (warp & 1) .., columns 32 (warp >> 1) ..)
#pragma unroll
        for (int ks = 0; ks < kHeadRays / 16; ks++) {
            uint32_t ah[4], al[4];
            ld_at(s.xt_h, 16 * (warp & 1), 16 * ks, ah);
            ld_at(s.xt_l, 16 * (warp & 1), 16 * ks, al);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int n0 = 32 * (warp >> 1) + 8 * q;
                const uint32_t bh0 = ld2(&s.z1t_h[n0 + g][16 * ks + 2 * t]);
                const uint32_t bh1 = ld2(&s.z1t_h[n0 + g][16 * ks + 8 + 2 * t]);
                const uint32_t bl0 = ld2(&s.z1t_l[n0 + g][16 * ks + 2 * t]);
                const uint32_t bl1 = ld2(&s.z1t_l[n0 + g][16 * ks + 8 + 2 * t]);
                mma16816(aw1[q], ah, bh0, bh1);
                mma16816(aw1[q], ah, bl0, bl1);
                mma16816(aw1[q], al, bh0, bh1);
            }
        }
        // dW3 (64 x 2, one entry per thread), b1 / b2 (one unit per thread), b3
        {
            const int i = tid >> 1, k = tid & 1;
            float acc = 0.f;
#pragma unroll 8
            for (int r = 0; r < kHeadRays; r++) acc += s.h2[r][i] * s.dO[r][k];
            aw3 += acc;
            const bf16(*th)[kPR] = tid < kHHid ? s.z1t_h : s.z2t_h;
            const bf16(*tl)[kPR] = tid < kHHid ? s.z1t_l : s.z2t_l;
            const int u = tid & (kHHid - 1);
            float sb = 0.f;
#pragma unroll 8
            for (int r = 0; r < kHeadRays; r++) sb += __bfloat162float(th[u][r]) + __bfloat162float(tl[u][r]);
            ab += sb;
            if (tid < kHOut) {
                float s3 = 0.f;
                for (int r = 0; r < kHeadRays; r++) s3 += s.dO[r][tid];
                ab3 += s3;
            }
        }
    }
    // flush: W1 | b1 | W2 | b2 | W3 | b3
    float* gW1p = grad;
    float* gb1p = grad + kW1;
    float* gW2p = gb1p + kHHid;
    float* gb2p = gW2p + kW2;
    float* gW3p = gb2p + kHHid;
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const int i = 16 * warp + g, j = 8 * nt + 2 * t;
        atomicAdd(gW2p + i * kHHid + j, aw2[nt][0]);
        atomicAdd(gW2p + i * kHHid + j + 1, aw2[nt][1]);
        atomicAdd(gW2p + (i + 8) * kHHid + j, aw2[nt][2]);
        atomicAdd(gW2p + (i + 8) * kHHid + j + 1, aw2[nt][3]);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const int i = 16 * (warp & 1) + g, j = 32 * (warp >> 1) + 8 * q + 2 * t;
        atomicAdd(gW1p + i * kHHid + j, aw1[q][0]);
        atomicAdd(gW1p + i * kHHid + j + 1, aw1[q][1]);
        atomicAdd(gW1p + (i + 8) * kHHid + j, aw1[q][2]);
        atomicAdd(gW1p + (i + 8) * kHHid + j + 1, aw1[q][3]);
    }
    atomicAdd(gW3p + tid, aw3);
    if (tid < kHHid) atomicAdd(gb1p + tid, ab);
    else atomicAdd(gb2p + tid - kHHid, ab);
    if (tid < kHOut) atomicAdd(gW3p + kW3 + tid, ab3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0 && loss) atomicAdd(loss, lsum);
}

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

size_t head_train_smem() { return sizeof(HeadTrainSmem); }

void launch_head_fwd(const float* x, int64_t R, const HeadW& hw, float* out, cudaStream_t st) {
    if (R <= 0) return;
    int64_t blocks = ((R + 15) / 16 + kHeadWarps - 1) / kHeadWarps;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_head_fwd<<<(unsigned)blocks, kHeadThreads, 0, st>>>(x, R, hw, out);
}

void launch_head_train(const float* x, int64_t R, const HeadW& hw, const float* y_int, const float* y_drop, float lam_i,
                       float lam_d, float* grad, float* loss, float* dx, cudaStream_t st) {
    if (R <= 0) return;
    const size_t sm = sizeof(HeadTrainSmem);
    cudaFuncSetAttribute(k_head_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int per_sm = 1, dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_head_train, kHeadThreads, sm);
    if (per_sm < 1) per_sm = 1;
    int64_t blocks = (R + kHeadRays - 1) / kHeadRays;
    if (blocks > (int64_t)sms * per_sm) blocks = (int64_t)sms * per_sm;
    k_head_train<<<(unsigned)blocks, kHeadThreads, sm, st>>>(x, R, hw, y_int, y_drop, lam_i, lam_d, grad, loss, dx);
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
