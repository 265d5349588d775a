// umma.cuh -- fifth-generation tensor-core helpers (tcgen05, sm_100a/sm_103a): shared-memory
// matrix descriptors for the canonical no-swizzle layouts, the kind::f16 instruction
// descriptor, MMA issue and commit, bounded mbarrier waits, Tensor Memory allocation and
// loads.
//
// Operand layout (16-bit elements, no swizzle).  A matrix is tiled into core matrices of
// 8 rows x 16 bytes.  K-major: a core holds 8 rows of 8 consecutive K elements; MN-major:
// 8 K rows of 8 consecutive M (or N) elements.  The descriptor gives the start address, the
// byte stride between cores adjacent along K (LBO) and between cores adjacent along M or N
// (SBO).  A buffer whose element (r, c) -- r = one operand dimension, c = the other, c
// contiguous within 16 bytes -- sits at (r / 8) * RS + (c / 8) * 128 + (r % 8) * 16 +
// (c % 8) * 2 serves both as a K-major operand (rows r = M or N, columns c = K: LBO = 128,
// SBO = RS) and as an MN-major one (c = M or N, r = K: LBO = RS, SBO = 128).
//
// Accumulators: an M = 128 product puts row m in TMEM lane m; M = 64 puts row m in lane
// 32 (m / 16) + m % 16 (each warp's 32-lane quarter holds 16 rows in its first 16 lanes).
#pragma once
#include <cstdint>

namespace splat {
namespace umma {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, c) in a buffer of the layout above with row-group stride rs.
__host__ __device__ constexpr int off(int r, int c, int rs) { return (r >> 3) * rs + (c >> 3) * 128 + (r & 7) * 16 + (c & 7) * 2; }

__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);   // version 1, no swizzle
}
// K step ks (16 K elements = two cores) of a buffer with row-group stride rs: as a K-major
// operand (rows = M/N) or as an MN-major one (rows = K).
__device__ __forceinline__ uint64_t desc_k(uint32_t base, int rs, int ks) { return desc(base + ks * 256, 128, rs); }
__device__ __forceinline__ uint64_t desc_mn(uint32_t base, int rs, int ks) { return desc(base + ks * 2 * rs, rs, 128); }
// The descriptor of K step ks from that of step 0: only the start address (the low field,
// in 16-byte units) moves, by 256 bytes (K-major) or 2 rs bytes (MN-major) per step; the
// field does not carry for addresses inside the 256 KB shared window.
__device__ __forceinline__ uint64_t step_k(uint64_t d0, int ks) { return d0 + (uint64_t)(ks * (256 >> 4)); }
__device__ __forceinline__ uint64_t step_mn(uint64_t d0, int rs, int ks) { return d0 + (uint64_t)(ks * ((2 * rs) >> 4)); }

// kind::f16 instruction descriptor: BF16 A and B, FP32 accumulator, M x N, majors.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A B, issued by one thread.
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"((uint32_t)accumulate));
}
// The mbarrier receives one arrival when every MMA this thread issued before has completed.
__device__ __forceinline__ void commit(uint64_t* mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Waits for the phase of the given parity; false if it did not complete within the limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit = 1u << 24) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < limit; it++) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(mbar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Generic-proxy shared-memory writes become visible to the tensor core.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Tensor Memory: one warp allocates ncols (a power of two >= 32) and later frees them.
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst_smem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 16 consecutive FP32 columns of this thread's lane (the warp's quarter of the lanes).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t u[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
          "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; j++) v[j] = __uint_as_float(u[j]);
}
__device__ __forceinline__ void tmem_ld2(uint32_t taddr, float (&v)[2]) {
    uint32_t u0, u1;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(u0), "=r"(u1) : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    v[0] = __uint_as_float(u0);
    v[1] = __uint_as_float(u1);
}

}  // namespace umma
}  // namespace splat
