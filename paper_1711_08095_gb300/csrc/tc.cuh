// Blackwell tensor-core helpers (tcgen05 + TMEM, inline PTX) for BF16 x BF16 -> FP32 products
// with both operands in shared memory in the no-swizzle canonical K-major layout.
//
// K-major canonical layout: the operand is cut into core matrices of 8 rows x 16 bytes
// (8 x 8 BF16).  Element (row r, k) of an operand with K elements per row sits at byte
//   ((r / 8) * (K / 8) + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2.
// In the matrix descriptor, the leading-dimension byte offset is the step between core
// matrices adjacent along K (128 B) and the stride-dimension byte offset the step between
// 8-row groups ((K / 8) * 128 B).  One MMA of kind::f16 consumes K = 16, i.e. two core
// matrices along K, so the k-th slice starts 256 * k bytes further.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace snect {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int kmajor_off(int r, int k, int K) {
    return ((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor: start address, leading / stride byte offsets, version 1,
// no swizzle
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D[tmem] (+)= A[128 x K] B[N x K]^T, K a multiple of 16; issued by one thread
__device__ __forceinline__ void mma_kmajor(uint32_t tmem, uint32_t a_smem, uint32_t b_smem, int K, int N,
                                           bool accumulate) {
    const uint32_t sbo = (uint32_t)(K / 8) * 128;
    const uint32_t id = idesc_bf16(128, N);
    for (int kc = 0; kc < K / 16; ++kc) {
        const uint64_t da = desc(a_smem + kc * 256, 128, sbo);
        const uint64_t db = desc(b_smem + kc * 256, 128, sbo);
        const uint32_t acc = (accumulate || kc > 0) ? 1u : 0u;
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(id), "r"(acc));
    }
}

__device__ __forceinline__ void commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
}

// waits for phase `phase` of the barrier; gives up after a bounded number of polls and
// returns false
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t phase) {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 24) && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(phase));
    }
    return done != 0;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;"); }

// 16 consecutive FP32 columns of this thread's TMEM lane (warp w reads lanes 32 (w % 4) ..)
__device__ __forceinline__ void ld16(uint32_t taddr, float *out) {
    uint32_t v[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 16; ++j) out[j] = __uint_as_float(v[j]);
}

}  // namespace tc
}  // namespace snect
