// umma_util.cuh -- inline-PTX helpers for the 5th-generation tensor cores (tcgen05, sm_100+ /
// sm_103a): tensor-memory allocation, shared-memory matrix descriptors, the BF16 MMA with an
// FP32 accumulator in tensor memory, its completion on an mbarrier, and the accumulator read-back.
//
// Conventions (PTX ISA, tcgen05 section):
// - An MMA of shape M x N x K computes D[M][N] (+)= A[M][K] B[N][K]^T; both operands are read
//   from shared memory through 64-bit matrix descriptors, D lives in tensor memory (TMEM).
// - For cta_group::1 and M = 128, row i of D is TMEM lane i and column j of D is TMEM column
//   (base + j), one 32-bit FP32 value per cell. Warp w of the CTA may read lanes 32 (w % 4) ..
//   32 (w % 4) + 31 only.
// - Operand layout used here: K-major without swizzle. The unit is the "core matrix": 8 rows of
//   16 bytes (8 BF16 values along K), stored as 128 contiguous bytes. The descriptor's leading
//   byte offset (LBO) is the distance between core matrices adjacent along K, the stride byte
//   offset (SBO) the distance between core matrices adjacent along M (or N). Start addresses
//   and both offsets are multiples of 16 bytes.
#pragma once

#include <stdint.h>

namespace bsk {

// Instruction descriptor of tcgen05.mma.kind::f16 for BF16 A and B, FP32 D, both operands
// K-major, dense, no negation: D format at bits 4-5 (1 = F32), A format at 7-9 and B format at
// 10-12 (1 = BF16), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t umma_idesc_bf16_f32(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle: start address >> 4 at bits 0-13, LBO >> 4 at
// bits 16-29, SBO >> 4 at bits 32-45, the fixed value 0b001 at bits 46-48, base offset 0,
// relative LBO mode, swizzle mode 0 (none) at bits 61-63.
__device__ __forceinline__ uint64_t umma_desc_noswizzle(uint32_t smem_addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((smem_addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Allocates ncols TMEM columns (a power of two >= 32) for the CTA; the whole warp executes it.
// The TMEM address is written to the shared-memory word dst. The permit to allocate again is
// given up at once, so that other CTAs on the SM are never kept waiting by this one.
__device__ __forceinline__ void tmem_alloc_warp(uint32_t* dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Frees the columns of tmem_alloc_warp; executed by the warp that allocated them.
__device__ __forceinline__ void tmem_dealloc_warp(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Orders tcgen05 operations before (after) a thread synchronisation (barrier or mbarrier wait).
__device__ __forceinline__ void tc_fence_before_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after_sync()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D (+)= A B^T with BF16 operands in shared memory and the FP32 accumulator at TMEM address
// tmem_d; accumulate = 0 overwrites D. Issued by a single thread; asynchronous.
__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Makes the mbarrier bar track the completion of every tcgen05 operation this thread issued
// before (one arrival when they are all done).
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(bar)))
                 : "memory");
}

// Reads 16 consecutive 32-bit TMEM columns of this thread's lane (shape 32x32b, 16 repeats):
// lane l of the warp gets row (taddr lane + l), columns taddr column .. + 15. The wait for the
// load is in the same statement, so that no use of v can be scheduled before it.
__device__ __forceinline__ void tmem_ld_32x32b_x16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

}  // namespace bsk
