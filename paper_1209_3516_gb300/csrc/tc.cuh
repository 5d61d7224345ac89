// tc.cuh -- 5th-generation tensor core (tcgen05) building blocks for sm_103a.
//
// Thin inline-PTX wrappers: tensor memory (TMEM) allocation, stores from and
// loads into registers, the MMA with A in TMEM and B in shared memory, its
// commit to an mbarrier, the ordering fences, and the shared-memory matrix and
// instruction descriptors.  Conventions used by the kernels here:
//   - one CTA of 4 warps (128 threads) owns an allocation of TMEM columns;
//     warp w may access TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 only;
//   - a TMEM address is (lane << 16) | column;
//   - MMAs are kind::f16 with BF16 operands, FP32 accumulation, M = 128 rows
//     (one TMEM lane per row), N = 32 columns, K = 16 per instruction;
//   - A (M x K) sits in TMEM, two BF16 per 32-bit column (the lower-index k in
//     the low half); B (K x N) sits in shared memory in the no-swizzle
//     "MN-major" canonical layout: 8 x 8 core matrices of 128 contiguous bytes
//     (one 16-byte row of 8 N-consecutive values per k), core matrices
//     adjacent in K at the leading-dimension byte offset, adjacent in N at the
//     stride-dimension byte offset.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fmm {
namespace tc {

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Allocate ncols (a power of two >= 32) TMEM columns; the base address is
// written to *dst (shared memory).  Whole warp, converged.
__device__ __forceinline__ void alloc(unsigned *dst, unsigned ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void relinquish() { asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void dealloc(unsigned taddr, unsigned ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 lanes x 256 bits: thread t writes lanes base + t/4 (r0, r1) and
// base + t/4 + 8 (r2, r3), columns 2 (t % 4) (r0, r2) and 2 (t % 4) + 1 (r1, r3).
__device__ __forceinline__ void st_16x256b(unsigned taddr, unsigned r0, unsigned r1, unsigned r2, unsigned r3)
{
    asm volatile("tcgen05.st.sync.aligned.16x256b.x1.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(r0), "r"(r1),
                 "r"(r2), "r"(r3)
                 : "memory");
}
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 32 lanes x 32 bits, 16 columns: thread t reads lane base + t, columns c .. c + 15.
__device__ __forceinline__ void ld_32x32b_x16(unsigned taddr, float *v)
{
    unsigned r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// D (TMEM) = A (TMEM) B (shared memory) + (accumulate ? D : 0); one thread issues.
__device__ __forceinline__ void mma_ts(unsigned d_tmem, unsigned a_tmem, uint64_t b_desc, unsigned idesc, bool accumulate)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
                 "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"((unsigned)accumulate)
                 : "memory");
}
// Arrive (once) on an mbarrier when every MMA this thread issued so far has completed.
__device__ __forceinline__ void commit(unsigned long long *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
                 : "memory");
}

// Shared-memory matrix descriptor, no swizzle: start address, leading- and
// stride-dimension byte offsets (multiples of 16), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(const void *p, unsigned lbo, unsigned sbo)
{
    const uint64_t a = smem_addr(p);
    return ((a & 0x3FFFFull) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 D, BF16 A and B, A K-major, B
// MN-major, dense, M x N.
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

}  // namespace tc
}  // namespace fmm
