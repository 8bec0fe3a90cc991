// umma.cuh -- fifth-generation tensor-core building blocks (tcgen05, sm_103a) for the learned
// edge-scoring network: tensor-memory allocation, BF16 MMAs with FP32 accumulators in tensor
// memory, their completion through an mbarrier, and the read-back of accumulator rows.
//
// Operands sit in shared memory in the canonical layouts without swizzle, in core matrices of 128
// contiguous bytes.  K-major: a core matrix is 8 rows (of M or N) x 16 bytes (8 BF16 along K).
// MN-major: 8 rows along K x 16 bytes (8 BF16 along M or N).  Either way the core matrix of M/N
// group g and K group c starts at byte g * SBO + c * LBO; every tile here uses LBO = 128 (the K
// groups of one M/N group adjacent) and SBO = 128 * (K groups in the tile).
//
// Accumulator layout for M = 128 with one CTA: row i of D in tensor-memory lane i, column j of D in
// column (base + j).  Warp w of the CTA reads lanes 32w .. 32w + 31.
#pragma once

#include <stdint.h>

namespace umma {

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading byte offset >> 4
// (bits 16-29), stride byte offset >> 4 (bits 32-45), descriptor version 1 (bits 46-47), base
// offset 0, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9 and 10-12 =
// 1), A and B K-major (bits 15, 16 = 0) or MN-major (= 1), N >> 3 in bits 17-22, M >> 4 in bits
// 24-28.
template <int M, int N, bool A_MN = false, bool B_MN = false>
struct IdescBf16 {
    static_assert(M == 128, "one-CTA tiles of 128 rows");
    static_assert(N % 16 == 0 && N >= 16 && N <= 256, "N for M = 128");
    static constexpr uint32_t value = (1u << 4) | (1u << 7) | (1u << 10) | ((A_MN ? 1u : 0u) << 15) |
                                      ((B_MN ? 1u : 0u) << 16) | ((uint32_t)(N >> 3) << 17) |
                                      ((uint32_t)(M >> 4) << 24);
};

// Whole warp: allocate `ncols` tensor-memory columns (a power of two >= 32); the base address is
// written to *slot.  The CTA allocates once, so it gives up its allocation permit right away.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Whole warp: free what tmem_alloc allocated.
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Shared-memory writes of this thread become visible to the tensor core's (async proxy) reads.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// One thread: D (tensor memory) = A B (+ D when accumulate), A M x 16 and B N x 16, both K-major.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// The issuing thread: one arrival on *bar once every MMA it issued before has completed.
__device__ __forceinline__ void commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Waits until the phase of parity `parity` of *bar has completed; gives up (false) after
// `limit_ns` nanoseconds of the global timer.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    const uint32_t a = smem_addr(bar);
    const uint64_t deadline_ns = now_ns() + limit_ns;
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if (now_ns() > deadline_ns) return false;
    }
}

// Whole warp: 32 consecutive accumulator columns of this thread's lane (lane quarter of the warp,
// column offset in taddr's low 16 bits), waiting for the load inside the same statement so that
// no use of the registers can be scheduled before it.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace umma
