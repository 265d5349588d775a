// head.cu -- the per-ray lidar decoder: rendered features + ray direction -> 64 -> 64 -> 2
// (intensity logit, ray-drop logit).  Paper Sec. 3.3 (features concatenated with the ray
// direction, decoded by a small MLP to intensity and ray-drop probability), App. B (a
// lightweight two-hidden-layer MLP; loss weights lambda_intens = 1, lambda_raydrop = 0.1
// in Eq. loss_fn).
//
// Weights are stored in BF16 (W1 | W2 | W3 packed) with FP32 biases and FP32 master copies
// for the optimiser; every product is accumulated in FP32 on the FMA pipe (activations
// stay FP32, so the decoder's error is that of FP32 accumulation, not of BF16 operands).
// Each block converts the weights to FP32 in shared memory once; a thread owns one ray.
// The training kernel runs the per-ray forward and backward, then forms the weight
// gradients of a 128-ray tile as tile-wide contractions out of shared memory, keeping
// them in registers across a persistent grid and flushing once per block.
#include <cuda_bf16.h>

#include "types.cuh"

namespace splat {

constexpr int kHIn = 32, kHHid = 64, kHOut = 2;
constexpr int kW1 = kHIn * kHHid, kW2 = kHHid * kHHid, kW3 = kHHid * kHOut;
constexpr int kHeadParams = kW1 + kHHid + kW2 + kHHid + kW3 + kHOut;   // W1 b1 W2 b2 W3 b3
constexpr int kHeadTile = 128;

struct HeadSmemW {
    float W1[kW1];
    float W2[kW2];
    float W3[kW3];
    float b1[kHHid], b2[kHHid], b3[kHOut];
};

__device__ __forceinline__ float bf16_to_f32(uint16_t u) { return __uint_as_float(((uint32_t)u) << 16); }

__device__ __forceinline__ void load_head_weights(HeadSmemW& s, const HeadW& hw) {
    for (int i = threadIdx.x; i < kW1 + kW2 + kW3; i += blockDim.x) {
        const float v = bf16_to_f32(hw.w[i]);
        if (i < kW1) s.W1[i] = v;
        else if (i < kW1 + kW2) s.W2[i - kW1] = v;
        else s.W3[i - kW1 - kW2] = v;
    }
    for (int i = threadIdx.x; i < 2 * kHHid + kHOut; i += blockDim.x) {
        const float v = hw.b[i];
        if (i < kHHid) s.b1[i] = v;
        else if (i < 2 * kHHid) s.b2[i - kHHid] = v;
        else s.b3[i - 2 * kHHid] = v;
    }
}

__device__ __forceinline__ void load_x(const float* x, int64_t r, float (&xr)[kHIn]) {
    const float4* p = reinterpret_cast<const float4*>(x + r * kHIn);
#pragma unroll
    for (int k = 0; k < kHIn / 4; k++) {
        const float4 v = p[k];
        xr[4 * k] = v.x;
        xr[4 * k + 1] = v.y;
        xr[4 * k + 2] = v.z;
        xr[4 * k + 3] = v.w;
    }
}

// h1 = relu(W1^T x + b1)
__device__ __forceinline__ void layer1(const HeadSmemW& s, const float (&xr)[kHIn], float (&h1)[kHHid]) {
#pragma unroll
    for (int j = 0; j < kHHid; j++) h1[j] = s.b1[j];
#pragma unroll 4
    for (int i = 0; i < kHIn; i++) {
        const float xi = xr[i];
#pragma unroll
        for (int j = 0; j < kHHid; j++) h1[j] += xi * s.W1[i * kHHid + j];
    }
#pragma unroll
    for (int j = 0; j < kHHid; j++) h1[j] = fmaxf(h1[j], 0.f);
}

// o = W3^T relu(W2^T h1 + b2) + b3, one hidden unit at a time; also returns the active mask.
__device__ __forceinline__ void layer23(const HeadSmemW& s, const float (&h1)[kHHid], float& o0, float& o1,
                                        uint64_t& mask, float* h2_out) {
    o0 = s.b3[0];
    o1 = s.b3[1];
    mask = 0;
#pragma unroll 2
    for (int j = 0; j < kHHid; j += 4) {
        float z[4];
#pragma unroll
        for (int q = 0; q < 4; q++) z[q] = s.b2[j + q];
#pragma unroll
        for (int i = 0; i < kHHid; i++) {
            const float hi = h1[i];
#pragma unroll
            for (int q = 0; q < 4; q++) z[q] += hi * s.W2[i * kHHid + j + q];
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const float h2 = fmaxf(z[q], 0.f);
            if (z[q] > 0.f) mask |= (uint64_t)1 << (j + q);
            if (h2_out) h2_out[j + q] = h2;
            o0 += h2 * s.W3[(j + q) * kHOut];
            o1 += h2 * s.W3[(j + q) * kHOut + 1];
        }
    }
}

__global__ void __launch_bounds__(256) k_head_fwd(const float* __restrict__ x, int64_t R, HeadW hw,
                                                  float* __restrict__ out) {
    __shared__ HeadSmemW s;
    load_head_weights(s, hw);
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < R; r += (int64_t)gridDim.x * blockDim.x) {
        float xr[kHIn], h1[kHHid];
        load_x(x, r, xr);
        layer1(s, xr, h1);
        float o0, o1;
        uint64_t mask;
        layer23(s, h1, o0, o1, mask, nullptr);
        reinterpret_cast<float2*>(out)[r] = make_float2(o0, o1);
    }
}

struct HeadTrainSmem {
    HeadSmemW w;
    float X[kHeadTile][kHIn];
    float H1[kHeadTile][kHHid];
    float A[kHeadTile][kHHid];     // h2, then dZ1 (relu'(z1) * dh1)
    float DZ2[kHeadTile][kHHid];
    float DO[kHeadTile][kHOut];
    float red[kHeadTile / 32];
};

// Loss lam_i mean (sigmoid(o0) - y_int)^2 + lam_d mean BCE(o1, y_drop) over R rays; adds
// its gradients to grad (W1 b1 W2 b2 W3 b3, FP32) and, if dx is given, writes dL/dx.
__global__ void __launch_bounds__(kHeadTile) k_head_train(const float* __restrict__ x, int64_t R, HeadW hw,
                                                         const float* __restrict__ y_int,
                                                         const float* __restrict__ y_drop, float lam_i, float lam_d,
                                                         float* __restrict__ grad, float* loss, float* __restrict__ dx) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    HeadTrainSmem& s = *reinterpret_cast<HeadTrainSmem*>(smem_raw);
    load_head_weights(s.w, hw);
    const int t = threadIdx.x;
    // register accumulators of this thread's share of the weight gradients
    float gW1[kW1 / kHeadTile], gW2[kW2 / kHeadTile], gW3 = 0.f, gb = 0.f, gb3a = 0.f, gb3b = 0.f;
#pragma unroll
    for (int k = 0; k < kW1 / kHeadTile; k++) gW1[k] = 0.f;
#pragma unroll
    for (int k = 0; k < kW2 / kHeadTile; k++) gW2[k] = 0.f;
    float lsum = 0.f;
    const float invR = 1.f / (float)R;
    const int64_t ntiles = (R + kHeadTile - 1) / kHeadTile;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r = tile * kHeadTile + t;
        const bool valid = r < R;
        __syncthreads();   // weights loaded / previous tile's contractions done
        float xr[kHIn], h1[kHHid];
        if (valid) load_x(x, r, xr);
        else {
#pragma unroll
            for (int i = 0; i < kHIn; i++) xr[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < kHIn; i++) s.X[t][i] = xr[i];
        layer1(s.w, xr, h1);
#pragma unroll
        for (int j = 0; j < kHHid; j++) s.H1[t][j] = h1[j];
        float o0, o1;
        uint64_t mask;
        layer23(s.w, h1, o0, o1, mask, s.A[t]);
        float d0 = 0.f, d1 = 0.f;
        if (valid) {
            const float sg = 1.f / (1.f + __expf(-o0));
            const float e = sg - y_int[r];
            const float y = y_drop[r];
            const float bce = fmaxf(o1, 0.f) - o1 * y + log1pf(__expf(-fabsf(o1)));
            lsum += lam_i * e * e * invR + lam_d * bce * invR;
            d0 = lam_i * 2.f * e * sg * (1.f - sg) * invR;
            d1 = lam_d * (1.f / (1.f + __expf(-o1)) - y) * invR;
        }
        s.DO[t][0] = d0;
        s.DO[t][1] = d1;
        gb3a += d0;
        gb3b += d1;
        // dZ2 = relu'(z2) * (W3 dO)
#pragma unroll
        for (int j = 0; j < kHHid; j++) {
            const float v = s.w.W3[j * kHOut] * d0 + s.w.W3[j * kHOut + 1] * d1;
            s.DZ2[t][j] = ((mask >> j) & 1) ? v : 0.f;
        }
        __syncthreads();
        // dW3 (64 x 2) and the biases: one entry per thread for this tile (h2 in A)
        {
            const int i = t >> 1, k = t & 1;   // 128 threads <-> 64 x 2 entries
            float acc = 0.f;
#pragma unroll 8
            for (int rr = 0; rr < kHeadTile; rr++) acc += s.A[rr][i] * s.DO[rr][k];
            gW3 += acc;
        }
        __syncthreads();
        // dZ1 = relu'(z1) * (W2 dZ2), written over h2
        {
            float dz2[kHHid];
#pragma unroll
            for (int j = 0; j < kHHid; j++) dz2[j] = s.DZ2[t][j];
#pragma unroll 4
            for (int i = 0; i < kHHid; i++) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < kHHid; j++) acc += s.w.W2[i * kHHid + j] * dz2[j];
                s.A[t][i] = s.H1[t][i] > 0.f ? acc : 0.f;
            }
        }
        __syncthreads();
        if (dx && valid) {
            float dz1[kHHid];
#pragma unroll
            for (int j = 0; j < kHHid; j++) dz1[j] = s.A[t][j];
#pragma unroll 4
            for (int i = 0; i < kHIn; i++) {
                float acc = 0.f;
#pragma unroll
                for (int j = 0; j < kHHid; j++) acc += s.w.W1[i * kHHid + j] * dz1[j];
                dx[r * kHIn + i] = acc;
            }
        }
        // dW1 = X^T dZ1, dW2 = H1^T dZ2 over the tile; thread t owns entries t + 128 k
#pragma unroll
        for (int k = 0; k < kW1 / kHeadTile; k++) {
            const int e = t + kHeadTile * k, i = e / kHHid, j = e % kHHid;
            float acc = 0.f;
#pragma unroll 8
            for (int rr = 0; rr < kHeadTile; rr++) acc += s.X[rr][i] * s.A[rr][j];
            gW1[k] += acc;
        }
#pragma unroll
        for (int k = 0; k < kW2 / kHeadTile; k++) {
            const int e = t + kHeadTile * k, i = e / kHHid, j = e % kHHid;
            float acc = 0.f;
#pragma unroll 8
            for (int rr = 0; rr < kHeadTile; rr++) acc += s.H1[rr][i] * s.DZ2[rr][j];
            gW2[k] += acc;
        }
        // biases: b1 (threads 0..63 sum dZ1 columns), b2 (64..127 sum dZ2), b3 below
        {
            float acc = 0.f;
            if (t < kHHid)
#pragma unroll 8
            for (int rr = 0; rr < kHeadTile; rr++) acc += s.A[rr][t];
            else
#pragma unroll 8
            for (int rr = 0; rr < kHeadTile; rr++) acc += s.DZ2[rr][t - kHHid];
            gb += acc;
        }
    }
    __syncthreads();
    // flush: W1 | b1 | W2 | b2 | W3 | b3
    float* gW1p = grad;
    float* gb1p = grad + kW1;
    float* gW2p = gb1p + kHHid;
    float* gb2p = gW2p + kW2;
    float* gW3p = gb2p + kHHid;
#pragma unroll
    for (int k = 0; k < kW1 / kHeadTile; k++) atomicAdd(gW1p + t + kHeadTile * k, gW1[k]);
#pragma unroll
    for (int k = 0; k < kW2 / kHeadTile; k++) atomicAdd(gW2p + t + kHeadTile * k, gW2[k]);
    atomicAdd(gW3p + t, gW3);
    if (t < kHHid) atomicAdd(gb1p + t, gb);
    else atomicAdd(gb2p + t - kHHid, gb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        gb3a += __shfl_xor_sync(0xffffffffu, gb3a, o);
        gb3b += __shfl_xor_sync(0xffffffffu, gb3b, o);
    }
    if ((t & 31) == 0) {
        atomicAdd(gW3p + kW3, gb3a);
        atomicAdd(gW3p + kW3 + 1, gb3b);
        if (loss) atomicAdd(loss, lsum);
    }
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

size_t head_train_smem() { return sizeof(HeadTrainSmem); }

void launch_head_fwd(const float* x, int64_t R, const HeadW& hw, float* out, cudaStream_t st) {
    if (R <= 0) return;
    int64_t blocks = (R + 255) / 256;
    if (blocks > 152 * 4) blocks = 152 * 4;
    k_head_fwd<<<(unsigned)blocks, 256, 0, st>>>(x, R, hw, out);
}

void launch_head_train(const float* x, int64_t R, const HeadW& hw, const float* y_int, const float* y_drop, float lam_i,
                       float lam_d, float* grad, float* loss, float* dx, cudaStream_t st) {
    if (R <= 0) return;
    const size_t sm = sizeof(HeadTrainSmem);
    cudaFuncSetAttribute(k_head_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int64_t blocks = (R + kHeadTile - 1) / kHeadTile;
    if (blocks > 152) blocks = 152;
    k_head_train<<<(unsigned)blocks, kHeadTile, sm, st>>>(x, R, hw, y_int, y_drop, lam_i, lam_d, grad, loss, dx);
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
