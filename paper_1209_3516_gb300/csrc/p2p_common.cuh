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

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

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
};

}  // namespace fmm
