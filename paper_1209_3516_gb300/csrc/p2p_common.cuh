// p2p_common.cuh -- source staging shared by the P2P kernels (forward and adjoint).
//
// The P2P list of a target leaf is held as runs of consecutive sibling leaves
// (one contiguous block of particles in one frame, the frame being the centre
// of the leaves' parent): a run record is (X_frame(S) - X_frame(T), first
// particle) and its end particle.  A warp walks an item's runs with a
// warp-uniform cursor and copies up to kS particles at a time into shared
// memory with cp.async, together with each particle's frame shift.
#pragma once

#include <cuda_runtime.h>

#include "device_util.cuh"

namespace fmm {

__device__ __forceinline__ int frame_of(const int *parent, int c) { return parent[c] >= 0 ? parent[c] : c; }

// Bulk-copy (TMA) staging: one lane issues one cp.async.bulk per contiguous
// run segment (16-byte aligned, a multiple of 16 bytes: float4 particles), the
// bytes counted on a per-buffer mbarrier that the consumers wait on.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *mbar, unsigned bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long *mbar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(mbar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *mbar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(mbar)), "r"(parity)
                 : "memory");
    return ok != 0u;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}
// Every lane waits for the phase of the given parity (a bounded number of
// polls); false for the whole warp if any lane gave up.
constexpr unsigned kMbarPolls = 1u << 20;
__device__ __forceinline__ bool mbar_wait_warp(unsigned long long *mbar, unsigned parity)
{
    bool done = false;
    for (unsigned i = 0; i < kMbarPolls && !done; ++i) done = mbar_try_wait(mbar, parity);
    return __all_sync(kFull, done);
}

// Warp-uniform cursor over an item's source runs, filling staging buffers.
struct RunCursor {
    int e, e1, o, pb, cnt;
    float shx, shy, shz;
    __device__ __forceinline__ void init(const unsigned *roff, int leaf_index, const float4 *run, const int *run_end)
    {
        e = (int)roff[leaf_index];
        e1 = (int)roff[leaf_index + 1];
        o = pb = cnt = 0;
        shx = shy = shz = 0.f;
        load(run, run_end);
    }
    __device__ __forceinline__ void load(const float4 *run, const int *run_end)
    {
        if (e < e1) {
            const float4 r = run[e];
            shx = r.x;
            shy = r.y;
            shz = r.z;
            pb = __float_as_int(r.w);
            cnt = run_end[e] - pb;
        }
    }
    // Copy up to kS particles into part (and, with kTwo, the same slots of src2
    // into part2) with cp.async, and their frame shift into shift; *self is set
    // when the copied particles overlap [tb0, tb1).  Returns the count.
    template <int kS, bool kTwo>
    __device__ __forceinline__ int stage(const float4 *run, const int *run_end, const float4 *pos, const float4 *src2,
                                         float4 *part, float4 *part2, float4 *shift, int tb0, int tb1, bool *self)
    {
        const int lane = (int)lane_id();
        int slots = 0;
        bool sf = false;
        while (slots < kS && e < e1) {
            const int m = min(cnt - o, kS - slots);
            const int begin = pb + o;
            sf |= begin < tb1 && begin + m > tb0;
            const float4 sh = make_float4(shx, shy, shz, 0.0f);
            for (int i = lane; i < m; i += 32) {
                cp_async16(part + slots + i, pos + begin + i);
                if (kTwo) cp_async16(part2 + slots + i, src2 + begin + i);
                shift[slots + i] = sh;
            }
            slots += m;
            o += m;
            if (o == cnt) {
                ++e;
                o = 0;
                load(run, run_end);
            }
        }
        *self = sf;
        return slots;
    }
    // The same walk with bulk copies: lane 0 issues one copy per run segment into
    // part and, last, the arrive on mbar (the buffer's previous contents have
    // been read by every lane: the caller has passed a __syncwarp).
    template <int kS>
    __device__ __forceinline__ int stage_bulk(const float4 *run, const int *run_end, const float4 *pos, float4 *part,
                                              float4 *shift, int tb0, int tb1, bool *self, unsigned long long *mbar)
    {
        const int lane = (int)lane_id();
        int slots = 0;
        bool sf = false;
        if (lane == 0) fence_proxy_async();
        while (slots < kS && e < e1) {
            const int m = min(cnt - o, kS - slots);
            const int begin = pb + o;
            sf |= begin < tb1 && begin + m > tb0;
            if (lane == 0) {
                mbar_expect_tx(mbar, (unsigned)m * 16u);
                bulk_g2s(part + slots, pos + begin, (unsigned)m * 16u, mbar);
            }
            const float4 sh = make_float4(shx, shy, shz, 0.0f);
            for (int i = lane; i < m; i += 32) shift[slots + i] = sh;
            slots += m;
            o += m;
            if (o == cnt) {
                ++e;
                o = 0;
                load(run, run_end);
            }
        }
        if (lane == 0) mbar_arrive(mbar);
        *self = sf;
        return slots;
    }
};

// Reduce-scatter 64 values across the warp by recursive halving: on return
// lane l holds entries 2l and 2l+1 of the warp-wide sums.
__device__ __forceinline__ void warp_reduce_scatter64(float *v)
{
    const unsigned lane = lane_id();
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        const int half = 32 >> step;          // values kept after this step
        const unsigned mask = 16u >> step;
        const bool upper = (lane & mask) != 0u;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(kFull, send, mask);
        }
    }
}

}  // namespace fmm
