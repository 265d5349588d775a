// mma.cuh -- warp-level tensor-core helpers shared by the decoder and the camera backward:
// mma.sync m16n8k16 with BF16 operands and FP32 accumulation, ldmatrix fragment loads,
// and the split of FP32 values into a BF16 high part and a BF16 residual.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

namespace splat {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ uint32_t bits2(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }
__device__ __forceinline__ uint32_t ld2(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// FP32 pair -> BF16 high parts and BF16 residuals (a = hi + lo to about 16 bits).
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    hi = bits2(h);
    lo = bits2(__floats2bfloat162_rn(a - hf.x, b - hf.y));
}

// d += A (16 x 16, row) * B (16 x 8, col): BF16 operands, FP32 accumulators.  Fragments:
// g = lane / 4, t = lane % 4; A regs (g, 2t..) (g+8, 2t..) (g, 2t+8..) (g+8, 2t+8..);
// B regs (k 2t.., n g) (k 2t+8.., n g); d (g, 2t) (g, 2t+1) (g+8, 2t) (g+8, 2t+1).
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Four 8 x 8 BF16 matrices from shared memory: lane i gives the address of row i % 8 of
// matrix i / 8 (16 bytes, 16-byte aligned); register j receives matrix j in the fragment
// layout (row g, columns 2t, 2t + 1).  The .trans form delivers each matrix transposed
// (rows 2t, 2t + 1 of column g).
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

}  // namespace splat
