// head_impl.cuh -- the per-ray lidar decoder's shared pieces (paper Sec. 3.3 decoder;
// App. B): layer sizes, the weights' shared-memory layouts, and the forward of one
// 16-ray tile on the tensor cores.  Used by the decoder kernels (head.cu) and by the
// lidar forward with the decoder fused into its epilogue.
#pragma once
#include <cuda_bf16.h>

#include "mma.cuh"
#include "types.cuh"

namespace splat {

constexpr int kHIn = 32, kHHid = 64, kHOut = 2;
constexpr int kW1 = kHIn * kHHid, kW2 = kHHid * kHHid, kW3 = kHHid * kHOut;
constexpr int kHeadParams = kW1 + kHHid + kW2 + kHHid + kW3 + kHOut;   // W1 b1 W2 b2 W3 b3
constexpr int kHeadWarps = 4;
constexpr int kHeadThreads = 32 * kHeadWarps;
constexpr int kHeadRays = 16 * kHeadWarps;   // rays per training-block iteration
constexpr int kP32 = 40;                      // padded row lengths (BF16 elements) of the shared
constexpr int kP64 = 72;                      // operands: conflict-free fragment loads
constexpr int kPR = kHeadRays + 8;            // transposed activations [unit][ray]

struct SplitA {   // an A fragment of split FP32 values
    uint32_t h[4], l[4];
};

// Weights in shared memory, in the layouts the fragments read: W^T [out][in] for the
// forward products (with the biases: all the forward needs), W [in][out] for the
// backward ones.
struct HeadSmemFwd {
    bf16 w1t[kHHid][kP32];
    bf16 w2t[kHHid][kP64];
    bf16 w3t[8][kP64];     // outputs 2..7 are zero (one 8-wide MMA tile)
    float b1[kHHid], b2[kHHid], b3[kHOut];
};
struct HeadSmemW : HeadSmemFwd {
    bf16 w1[kHIn][kP64];
    bf16 w2[kHHid][kP64];
    float w3[kHHid][kHOut];
};

// The forward weights and biases (any block size).
__device__ __forceinline__ void load_head_fwd_weights(HeadSmemFwd& s, const HeadW& hw) {
    const bf16* w = reinterpret_cast<const bf16*>(hw.w);
    for (int e = threadIdx.x; e < kW1; e += blockDim.x) s.w1t[e % kHHid][e / kHHid] = w[e];
    for (int e = threadIdx.x; e < kW2; e += blockDim.x) s.w2t[e % kHHid][e / kHHid] = w[kW1 + e];
    for (int e = threadIdx.x; e < 8 * kHHid; e += blockDim.x) {
        const int k = e / kHHid, i = e % kHHid;
        s.w3t[k][i] = k < kHOut ? w[kW1 + kW2 + i * kHOut + k] : __float2bfloat16_rn(0.f);
    }
    for (int e = threadIdx.x; e < 2 * kHHid + kHOut; e += blockDim.x) {
        const float v = hw.b[e];
        if (e < kHHid) s.b1[e] = v;
        else if (e < 2 * kHHid) s.b2[e - kHHid] = v;
        else s.b3[e - 2 * kHHid] = v;
    }
}

// Forward and backward weights.
__device__ __forceinline__ void load_head_weights(HeadSmemW& s, const HeadW& hw) {
    load_head_fwd_weights(s, hw);
    const bf16* w = reinterpret_cast<const bf16*>(hw.w);
    for (int e = threadIdx.x; e < kW1; e += blockDim.x) s.w1[e / kHHid][e % kHHid] = w[e];
    for (int e = threadIdx.x; e < kW2; e += blockDim.x) s.w2[e / kHHid][e % kHHid] = w[kW1 + e];
    for (int e = threadIdx.x; e < kHHid * kHOut; e += blockDim.x)
        s.w3[e / kHOut][e % kHOut] = __bfloat162float(w[kW1 + kW2 + e]);
}

// One C tile (n-tile nt of a 64-wide layer) -> the A fragment of the next layer.
__device__ __forceinline__ void c_to_a(const float (&d)[4], int nt, SplitA (&a)[4]) {
    const int ks = nt >> 1, r = (nt & 1) * 2;
    split_pair(d[0], d[1], a[ks].h[r], a[ks].l[r]);
    split_pair(d[2], d[3], a[ks].h[r + 1], a[ks].l[r + 1]);
}

// The forward of one 16-ray tile: x fragments in, H1 / H2 fragments, ReLU masks (bit
// 4 nt + e for accumulator e of n-tile nt) and the two outputs of rows g and g + 8 out
// (valid on lanes with t == 0).
struct HeadFwd {
    SplitA h1[4], h2[4];
    uint32_t m1, m2;
    float o[4];   // (o0, o1) of row g, (o0, o1) of row g + 8
};

__device__ __forceinline__ void head_forward_tile(const HeadSmemFwd& s, const SplitA (&xa)[2], HeadFwd& f) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    f.m1 = f.m2 = 0;
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const float ba = s.b1[8 * nt + 2 * t], bb = s.b1[8 * nt + 2 * t + 1];
        float d[4] = {ba, bb, ba, bb};
#pragma unroll
        for (int ks = 0; ks < 2; ks++) {
            const uint32_t b0 = ld2(&s.w1t[8 * nt + g][16 * ks + 2 * t]);
            const uint32_t b1 = ld2(&s.w1t[8 * nt + g][16 * ks + 8 + 2 * t]);
            mma16816(d, xa[ks].h, b0, b1);
            mma16816(d, xa[ks].l, b0, b1);
        }
#pragma unroll
        for (int e = 0; e < 4; e++) {
            if (d[e] > 0.f) f.m1 |= 1u << (4 * nt + e);
            else d[e] = 0.f;
        }
        c_to_a(d, nt, f.h1);
    }
#pragma unroll
    for (int nt = 0; nt < 8; nt++) {
        const float ba = s.b2[8 * nt + 2 * t], bb = s.b2[8 * nt + 2 * t + 1];
        float d[4] = {ba, bb, ba, bb};
#pragma unroll
        for (int ks = 0; ks < 4; ks++) {
            const uint32_t b0 = ld2(&s.w2t[8 * nt + g][16 * ks + 2 * t]);
            const uint32_t b1 = ld2(&s.w2t[8 * nt + g][16 * ks + 8 + 2 * t]);
            mma16816(d, f.h1[ks].h, b0, b1);
            mma16816(d, f.h1[ks].l, b0, b1);
        }
#pragma unroll
        for (int e = 0; e < 4; e++) {
            if (d[e] > 0.f) f.m2 |= 1u << (4 * nt + e);
            else d[e] = 0.f;
        }
        c_to_a(d, nt, f.h2);
    }
    const float b30 = t == 0 ? s.b3[0] : 0.f, b31 = t == 0 ? s.b3[1] : 0.f;
    float d[4] = {b30, b31, b30, b31};
#pragma unroll
    for (int ks = 0; ks < 4; ks++) {
        const uint32_t b0 = ld2(&s.w3t[g][16 * ks + 2 * t]);
        const uint32_t b1 = ld2(&s.w3t[g][16 * ks + 8 + 2 * t]);
        mma16816(d, f.h2[ks].h, b0, b1);
        mma16816(d, f.h2[ks].l, b0, b1);
    }
#pragma unroll
    for (int e = 0; e < 4; e++) f.o[e] = d[e];
}

// x rows r0 + g and r0 + g + 8 (zero past R) as split A fragments of the two k-steps;
// also returns the raw values (k-step ks, register q, element e) for transposed copies.
__device__ __forceinline__ void load_x_frags(const float* __restrict__ x, int64_t r0, int64_t R, SplitA (&xa)[2],
                                             float (&xv)[2][4][2]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int64_t ra = r0 + g, rb = r0 + g + 8;
#pragma unroll
    for (int ks = 0; ks < 2; ks++) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int64_t r = (q & 1) ? rb : ra;
            const int col = 16 * ks + ((q & 2) ? 8 : 0) + 2 * t;
            float2 v = make_float2(0.f, 0.f);
            if (r < R) v = *reinterpret_cast<const float2*>(x + r * kHIn + col);
            xv[ks][q][0] = v.x;
            xv[ks][q][1] = v.y;
            split_pair(v.x, v.y, xa[ks].h[q], xa[ks].l[q]);
        }
    }
}

// The A-fragment elements of a 16-ray input tile, as loaded (FP32 pairs).
__device__ __forceinline__ void load_x_raw(const float* __restrict__ x, int64_t r0, int64_t R, float2 (&v)[2][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int ks = 0; ks < 2; ks++) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int64_t r = r0 + g + ((q & 1) ? 8 : 0);
            const int col = 16 * ks + ((q & 2) ? 8 : 0) + 2 * t;
            v[ks][q] = r < R ? *reinterpret_cast<const float2*>(x + r * kHIn + col) : make_float2(0.f, 0.f);
        }
    }
}

}  // namespace splat
