// device_util.cuh -- small device helpers shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fmm {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Hardware reciprocal square root (SFU, ~2^-23 relative error), denormal inputs
// flushed to zero.  Callers pass normal positive numbers (or 0, giving +inf).
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <class T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Spread the low 21 bits of v so that bit b lands at bit 3b.
__host__ __device__ __forceinline__ uint64_t spread3(uint64_t v)
{
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x001f00000000ffffull;
    v = (v | (v << 16)) & 0x001f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Inverse of spread3: gather every third bit (starting at bit 0) into the low bits.
__host__ __device__ __forceinline__ uint32_t compact3(uint64_t v)
{
    v &= 0x1249249249249249ull;
    v = (v ^ (v >> 2)) & 0x10c30c30c30c30c3ull;
    v = (v ^ (v >> 4)) & 0x100f00f00f00f00full;
    v = (v ^ (v >> 8)) & 0x001f0000ff0000ffull;
    v = (v ^ (v >> 16)) & 0x001f00000000ffffull;
    v = (v ^ (v >> 32)) & 0x1fffffull;
    return (uint32_t)v;
}

// Warp-aggregated append of `val` (when pred) to buf[counter++] with a capacity check.
// Every lane of the warp must call it.  Overflowing entries are dropped and flagged;
// the counter still counts them so the host can size the next attempt.
template <class T>
__device__ __forceinline__ void warp_append(bool pred, const T &val, T *buf, unsigned long long cap,
                                            unsigned long long *counter, unsigned *overflow,
                                            unsigned bit)
{
    unsigned m = __ballot_sync(kFull, pred);
    if (m == 0u) return;
    int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (pred) {
        unsigned long long i = base + __popc(m & lanemask_lt());
        if (i < cap) buf[i] = val;
        else atomicOr(overflow, bit);
    }
}

// Asynchronous 16-byte global -> shared copies (cp.async, cached in L1 and L2),
// grouped by commit; wait_group 1 leaves the most recent group in flight.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

}  // namespace fmm
