// traverse.cu -- dual tree traversal (Algorithms 3 and 4) and list grouping.
//
// Algorithm 3: pop a pair (A, B); split the larger cell (A when B is a leaf,
// or when A is not a leaf and B_A > B_B; otherwise B, so ties split the source);
// Algorithm 4 for every child pair: both leaves -> P2P, MAC -> M2L, else push.
// MAC (Sec. 3.2): theta * |X_A - X_B| > B_A + B_B, in FP32 with one rounding
// per operation (the same decision an FP32 implementation of the definition
// takes).  The paper runs the traversal as tasks (TBB / OpenMP 3.0, Sec. 3.3);
// here it runs in two GPU stages:
//   1. breadth-first seeding rounds: one thread per (pair, child), until the
//      frontier holds about four pairs per resident warp of the device;
//   2. a persistent kernel: each warp claims seeds with an atomic counter and
//      runs the traversal below each seed depth first on a private stack in
//      shared memory, four pairs (32 child pairs) per step, for at most
//      kSeedBudget steps per seed; a warp whose budget runs out (or whose stack
//      is full) spills its remaining pairs to global memory, and the spilled
//      pairs seed another launch.  The budget keeps the launches balanced on
//      adaptive trees, where a few seeds own most of the traversal (the core of
//      a Plummer sphere): their subtrees are cut into pieces that every warp
//      shares in the next launch.  No warp ever waits on another.
// The emitted (target, source) pairs are then sorted by (target, source) so
// that every target cell owns a contiguous, ordered run of sources.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdio>

#include "device_util.cuh"
#include "fmm_internal.cuh"

namespace fmm {

constexpr unsigned kOvM2L = 1u, kOvP2P = 2u, kOvNext = 4u;
constexpr int kStackCap = 128;      // pairs per warp stack (24 bytes each)
constexpr int kStackWarps = 8;      // warps per block of the work-stack kernel
constexpr int kStackBlocksPerSM = 8;   // 64 resident warps per SM (24 KiB shared memory, <= 32 registers)
#ifndef FMM_SEED_BUDGET
#define FMM_SEED_BUDGET 128
#endif
#ifndef FMM_PASSES_PER_SYNC
#define FMM_PASSES_PER_SYNC 2
#endif
constexpr int kSeedBudget = FMM_SEED_BUDGET;   // steps per claimed seed before the rest is handed on
constexpr int kPassesPerSync = FMM_PASSES_PER_SYNC;   // work-stack passes back to back between host checks
static_assert(kPassesPerSync >= 1 && kPassesPerSync <= 8, "pass counters");
constexpr int kMaxStackPasses = 256;

struct Cell {
    float4 g;   // centre, radius
    int2 k;     // first child, child count (0 = leaf)
    int n;      // particles
};

__device__ __forceinline__ Cell load_cell(const float4 *geom, const int2 *kids, const int *pcnt, int c)
{
    Cell r;
    r.g = geom[c];
    r.k = kids[c];
    r.n = pcnt[c];
    return r;
}

__device__ __forceinline__ bool mac(const Cell &a, const Cell &b, float theta)
{
    const float dx = __fsub_rn(a.g.x, b.g.x), dy = __fsub_rn(a.g.y, b.g.y), dz = __fsub_rn(a.g.z, b.g.z);
    const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    const float R = __fsqrt_rn(r2);
    return __fmul_rn(theta, R) > __fadd_rn(a.g.w, b.g.w);
}

// Algorithm 4 outcome for the pair (a, b): 1 = P2P, 2 = M2L, 3 = push.  Both
// leaves go to P2P before the MAC is looked at, unless the M2L / P2P hybrid is
// on (hybrid_min >= 0): then a leaf pair that passes the MAC and holds at least
// hybrid_min particle pairs is an M2L pair.
__device__ __forceinline__ int interact(const Cell &a, const Cell &b, float theta, long long hybrid_min)
{
    if (a.k.y == 0 && b.k.y == 0) {
        if (hybrid_min >= 0 && (long long)a.n * (long long)b.n >= hybrid_min && mac(a, b, theta)) return 2;
        return 1;
    }
    return mac(a, b, theta) ? 2 : 3;
}

// Algorithm 3 split rule: true = split the target A.
__device__ __forceinline__ bool split_target(const Cell &A, const Cell &B)
{
    return B.k.y == 0 || (A.k.y != 0 && A.g.w > B.g.w);
}

// The emitted M2L and P2P pairs go to per-block regions of the list buffers:
// region r of a list holds cap entries from r cap on, counted in reg[r] (M2L)
// and reg[nreg + r] (P2P), one region per block of the work-stack kernel,
// which appends to it through a shared-memory counter; block b of a seeding
// round appends to region b mod nreg through global atomics.  (One global
// counter for all appends made the traversal wait on the serialised atomics.)
struct TravArgs {
    const float4 *geom;
    const int2 *kids;
    const int *pcnt;
    float theta;
    long long hybrid_min;   // < 0: Algorithm 4 as printed
    int2 *m2l;
    int2 *p2p;
    unsigned cap_m2l, cap_p2p;   // region capacities (multiples of 32)
    unsigned *reg;               // region counts, 2 nreg
    int nreg;
    int2 *next;
    unsigned long long next_cap;
    unsigned long long *n_next;   // count of pairs written to next (seeding round or work-stack pass)
    unsigned long long *claim;    // work-stack pass: next seed to claim
    TravCounters *ctr;
};

// Warp-aggregated append to a region with a 32-bit counter (global or shared
// memory); entries past the capacity are dropped and flagged, the counter
// still counts them.  Every lane of the warp calls it.
__device__ __forceinline__ void region_append(bool pred, int2 val, int2 *region, unsigned cap, unsigned *count,
                                              unsigned *overflow, unsigned bit)
{
    const unsigned m = __ballot_sync(kFull, pred);
    if (m == 0u) return;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(count, (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (pred) {
        const unsigned i = base + __popc(m & lanemask_lt());
        if (i < cap) region[i] = val;
        else atomicOr(overflow, bit);
    }
}

// Child pair j (0..7) of a popped pair; returns false when the split cell has fewer children.
__device__ __forceinline__ bool child_pair(const TravArgs &a, int2 pr, int j, int2 &np, Cell &ca, Cell &cb)
{
    const Cell A = load_cell(a.geom, a.kids, a.pcnt, pr.x);
    const Cell B = load_cell(a.geom, a.kids, a.pcnt, pr.y);
    if (split_target(A, B)) {
        if (j >= A.k.y) return false;
        np = make_int2(A.k.x + j, pr.y);
        ca = load_cell(a.geom, a.kids, a.pcnt, np.x);
        cb = B;
    } else {
        if (j >= B.k.y) return false;
        np = make_int2(pr.x, B.k.x + j);
        ca = A;
        cb = load_cell(a.geom, a.kids, a.pcnt, np.y);
    }
    return true;
}

// Seeding round: one thread per (frontier pair, child slot).  The frontier size
// is read from device memory (*nfront_p, at most the buffer capacity), the next
// frontier's size is counted into *nnext_p, so rounds run back to back without
// the host.
__global__ void k_dtt_round(const int2 *front, const unsigned long long *nfront_p, unsigned long long *nnext_p,
                            TravArgs a)
{
    const unsigned long long nfront = min(*nfront_p, a.next_cap);
    const unsigned long long total = nfront * 8ull;
    const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long w0 = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    for (unsigned long long base = w0 * 32ull; base < total; base += nwarps * 32ull) {
        const unsigned long long t = base + lane_id();
        int kind = 0;
        int2 np = make_int2(0, 0);
        if (t < total) {
            Cell ca, cb;
            if (child_pair(a, front[t >> 3], (int)(t & 7ull), np, ca, cb)) kind = interact(ca, cb, a.theta, a.hybrid_min);
        }
        const int rg = (int)(blockIdx.x % (unsigned)a.nreg);
        region_append(kind == 1, np, a.p2p + (size_t)rg * a.cap_p2p, a.cap_p2p, &a.reg[a.nreg + rg],
                      &a.ctr->overflow, kOvP2P);
        region_append(kind == 2, np, a.m2l + (size_t)rg * a.cap_m2l, a.cap_m2l, &a.reg[rg], &a.ctr->overflow,
                      kOvM2L);
        warp_append(kind == 3, np, a.next, a.next_cap, nnext_p, &a.ctr->overflow, kOvNext);
    }
}

// A stack entry of the work-stack kernel: the pair, both cells' children
// (first child << 4 | child count) and both radii, so that the split rule
// needs no load and one round of loads serves a step: the j-th child of the
// cell that is split and the other cell's centre (and particle count).
__device__ __forceinline__ int pack_kids(int2 k) { return (int)(((unsigned)k.x << 4) | (unsigned)k.y); }
__device__ __forceinline__ int2 unpack_kids(int v) { return make_int2((int)((unsigned)v >> 4), v & 15); }

// Persistent work-stack kernel; the seed count is read from device memory.
__global__ void __launch_bounds__(kStackWarps * 32, kStackBlocksPerSM) k_dtt_stack(const int2 *seeds,
                                                                                   const unsigned long long *nseeds_p,
                                                                                   TravArgs a)
{
    const unsigned long long nseeds = min(*nseeds_p, a.next_cap);
    __shared__ int4 stack[kStackWarps][kStackCap];     // a, b, packed children of a and b
    __shared__ float2 radii[kStackWarps][kStackCap];   // radius of a, of b
    __shared__ unsigned s_count[2];                    // this block's region counts (M2L, P2P)
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_count[0] = a.reg[blockIdx.x];
        s_count[1] = a.reg[a.nreg + blockIdx.x];
    }
    __syncthreads();
    int2 *const reg_m2l = a.m2l + (size_t)blockIdx.x * a.cap_m2l;
    int2 *const reg_p2p = a.p2p + (size_t)blockIdx.x * a.cap_p2p;
    const bool with_n = a.hybrid_min >= 0;   // particle counts matter only to the hybrid rule
    int4 *st = stack[w];
    float2 *sr = radii[w];
    int top = 0, steps = 0;
    for (;;) {
        if (top > 0 && steps >= kSeedBudget) {
            // budget used up: hand the remaining pairs to the next launch
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(a.n_next, (unsigned long long)top);
            base = __shfl_sync(kFull, base, 0);
            for (int i = (int)lane; i < top; i += 32) {
                if (base + i < a.next_cap) a.next[base + i] = make_int2(st[i].x, st[i].y);
                else atomicOr(&a.ctr->overflow, kOvNext);
            }
            top = 0;
            __syncwarp();
        }
        if (top == 0) {
            unsigned long long s = 0;
            if (lane == 0) s = atomicAdd(a.claim, 1ull);
            s = __shfl_sync(kFull, s, 0);
            if (s >= nseeds) break;
            if (lane == 0) {
                const int2 sd = seeds[s];
                st[0] = make_int4(sd.x, sd.y, pack_kids(a.kids[sd.x]), pack_kids(a.kids[sd.y]));
                sr[0] = make_float2(a.geom[sd.x].w, a.geom[sd.y].w);
            }
            top = 1;
            steps = 0;
            __syncwarp();
        }
        ++steps;
        const int npop = min(top, 4);
        top -= npop;
        const int p = (int)(lane >> 3), j = (int)(lane & 7u);
        int kind = 0;
        int2 np = make_int2(0, 0);
        Cell ca, cb;
        int4 pr = make_int4(0, 0, 0, 0);
        float2 rr = make_float2(0.f, 0.f);
        if (p < npop) {
            pr = st[top + p];
            rr = sr[top + p];
        }
        __syncwarp();   // every popped entry is read before pushes overwrite the slots
        if (p < npop) {
            Cell A, B;
            A.k = unpack_kids(pr.z);
            B.k = unpack_kids(pr.w);
            A.g.w = rr.x;
            B.g.w = rr.y;
            if (split_target(A, B)) {
                if (j < A.k.y) {
                    np = make_int2(A.k.x + j, pr.y);
                    ca.g = a.geom[np.x];
                    ca.k = a.kids[np.x];
                    ca.n = with_n ? a.pcnt[np.x] : 0;
                    cb.g = a.geom[pr.y];
                    cb.k = B.k;
                    cb.n = with_n ? a.pcnt[pr.y] : 0;
                    kind = interact(ca, cb, a.theta, a.hybrid_min);
                }
            } else if (j < B.k.y) {
                np = make_int2(pr.x, B.k.x + j);
                ca.g = a.geom[pr.x];
                ca.k = A.k;
                ca.n = with_n ? a.pcnt[pr.x] : 0;
                cb.g = a.geom[np.y];
                cb.k = a.kids[np.y];
                cb.n = with_n ? a.pcnt[np.y] : 0;
                kind = interact(ca, cb, a.theta, a.hybrid_min);
            }
        }
        region_append(kind == 1, np, reg_p2p, a.cap_p2p, &s_count[1], &a.ctr->overflow, kOvP2P);
        region_append(kind == 2, np, reg_m2l, a.cap_m2l, &s_count[0], &a.ctr->overflow, kOvM2L);
        const unsigned push = __ballot_sync(kFull, kind == 3);
        const int npush = __popc(push);
        if (top + npush <= kStackCap) {
            if (kind == 3) {
                const int slot = top + __popc(push & lanemask_lt());
                st[slot] = make_int4(np.x, np.y, pack_kids(ca.k), pack_kids(cb.k));
                sr[slot] = make_float2(ca.g.w, cb.g.w);
            }
            top += npush;
        } else {
            warp_append(kind == 3, np, a.next, a.next_cap, a.n_next, &a.ctr->overflow, kOvNext);
        }
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a.reg[blockIdx.x] = s_count[0];
        a.reg[a.nreg + blockIdx.x] = s_count[1];
    }
}

// Totals and largest region of both lists (one block of 256 threads).
__global__ void k_region_totals(int nreg, const unsigned *reg, TravCounters *ctr)
{
    __shared__ unsigned long long s_sum[2][8];
    __shared__ unsigned s_max[2][8];
    unsigned long long s0 = 0, s1 = 0;
    unsigned m0 = 0, m1 = 0;
    for (int r = threadIdx.x; r < nreg; r += blockDim.x) {
        s0 += reg[r];
        s1 += reg[nreg + r];
        m0 = max(m0, reg[r]);
        m1 = max(m1, reg[nreg + r]);
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    m0 = __reduce_max_sync(kFull, m0);
    m1 = __reduce_max_sync(kFull, m1);
    const int w = threadIdx.x >> 5;
    if (lane_id() == 0) {
        s_sum[0][w] = s0;
        s_sum[1][w] = s1;
        s_max[0][w] = m0;
        s_max[1][w] = m1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t0 = 0, t1 = 0;
        unsigned x0 = 0, x1 = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            t0 += s_sum[0][k];
            t1 += s_sum[1][k];
            x0 = max(x0, s_max[0][k]);
            x1 = max(x1, s_max[1][k]);
        }
        ctr->n_m2l = t0;
        ctr->n_p2p = t1;
        ctr->reg_max[0] = x0;
        ctr->reg_max[1] = x1;
    }
}

// ---------------------------------------------------------------------------
// list grouping
// ---------------------------------------------------------------------------
template <class K> __global__ void k_pack_pairs(const int2 *pairs, int64_t n, int cbits, K *keys)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int2 p = pairs[i];
    keys[i] = ((K)(unsigned)p.x << cbits) | (K)(unsigned)p.y;
}

template <class K> __global__ void k_unpack_sources(const K *keys, int64_t n, int cbits, int *src)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    src[i] = (int)(keys[i] & (((K)1 << cbits) - (K)1));
}

// off[c] = first entry whose target is >= c, for c = 0..ncells.
template <class K> __global__ void k_csr_offsets(const K *keys, int64_t n, int cbits, int ncells, int *off)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncells) return;
    const K v = (K)c << cbits;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    off[c] = (int)lo;
}

__global__ void k_pack_kids(int nc, const int *cbeg, const int *ccnt, int2 *kids)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < nc) kids[c] = make_int2(cbeg[c], ccnt[c]);
}

// Leaves in cell order, and the P2P particle-pair count sum n_T * n_S.
__global__ void k_leaf_list(int nc, const int *ccnt, int *leaf_list, unsigned *nleaves)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const bool leaf = c < nc && ccnt[c] == 0;
    const unsigned m = __ballot_sync(kFull, leaf);
    if (m == 0u) return;
    const int leader = __ffs(m) - 1;
    unsigned base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(nleaves, (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (leaf) leaf_list[base + __popc(m & lanemask_lt())] = c;
}

// A list as the traversal leaves it: region r holds cnt[r] pairs from r cap on.
struct RegionList {
    const int2 *pairs;
    const unsigned *cnt;
    unsigned cap;   // multiple of 32
    int nreg;
};

// Walk over a region list: block b takes regions b, b + gridDim.x, ..., its
// warps the 32-entry chunks of each; f(lane's pair, valid, region, index) is
// called by every lane of a chunk.
template <class F> __device__ __forceinline__ void for_each_chunk(const RegionList &L, F f)
{
    const unsigned lane = lane_id();
    for (int r = blockIdx.x; r < L.nreg; r += gridDim.x) {
        const unsigned n = min(L.cnt[r], L.cap);
        const int2 *pr = L.pairs + (size_t)r * L.cap;
        for (unsigned off = threadIdx.x - lane; off < n; off += blockDim.x) {
            const unsigned k = off + lane;
            const bool valid = k < n;
            const int2 p = valid ? pr[k] : make_int2(-1, 0);
            f(p, valid, r, k);
        }
    }
}

// dense[roff[r] + k] = pair k of region r
__global__ void k_compact_regions(RegionList L, const unsigned *roff, int2 *dense)
{
    for_each_chunk(L, [&](int2 p, bool valid, int r, unsigned k) {
        if (valid) dense[roff[r] + k] = p;
    });
}

// Radix form of the grouping (used only for a list with a repeated
// (target, source) pair, which the traversal does not emit): sort the (target, source) pairs by target, then
// source, packed as target << cbits | source (32-bit keys whenever
// 2 cbits <= 32), and split them into CSR form.
template <class K> static int group_list_radix_k(Handle &h, const int2 *pairs, int64_t n, int cbits, DevBuf &src,
                                                 DevBuf &off)
{
    const int nc = (int)h.ncells;
    FMM_TRY(h.lkeys.reserve(std::max<int64_t>(n, 1) * sizeof(K)));
    FMM_TRY(h.lkeys_alt.reserve(std::max<int64_t>(n, 1) * sizeof(K)));
    if (n > 0) {
        ++h.launches;
        k_pack_pairs<K><<<ceil_div(n, 256), 256, 0, h.stream>>>(pairs, n, cbits, h.lkeys.as<K>());
        K *k = h.lkeys.as<K>(), *ka = h.lkeys_alt.as<K>();
        if constexpr (sizeof(K) == 4) FMM_TRY(radix_sort_keys32(h, k, ka, n, 0, 2 * cbits));
        else FMM_TRY(radix_sort_keys(h, k, ka, n, 0, 2 * cbits));
        if (k != h.lkeys.as<K>()) std::swap(h.lkeys, h.lkeys_alt);
        ++h.launches;
        k_unpack_sources<K><<<ceil_div(n, 256), 256, 0, h.stream>>>(h.lkeys.as<K>(), n, cbits, src.as<int>());
    }
    ++h.launches;
    k_csr_offsets<K><<<ceil_div(nc + 1, 256), 256, 0, h.stream>>>(h.lkeys.as<K>(), n, cbits, nc, off.as<int>());
    FMM_CHECK_LAUNCH("group list (radix)");
    return FMM_OK;
}

static int group_list_radix(Handle &h, const RegionList &L, int64_t n, DevBuf &src, DevBuf &off)
{
    // the regions back to back first
    FMM_TRY(h.ldense.reserve(std::max<int64_t>(n, 1) * sizeof(int2) + (size_t)(L.nreg + 1) * sizeof(unsigned)));
    int2 *dense = h.ldense.as<int2>();
    unsigned *roff = reinterpret_cast<unsigned *>(dense + std::max<int64_t>(n, 1));
    FMM_TRY(scan_exclusive_u32(h, L.cnt, roff, L.nreg, nullptr));
    ++h.launches;
    k_compact_regions<<<L.nreg, 256, 0, h.stream>>>(L, roff, dense);
    const int2 *pairs = dense;
    int cbits = 1;
    while ((1ll << cbits) <= h.ncells) ++cbits;
    if (2 * cbits <= 32) return group_list_radix_k<uint32_t>(h, pairs, n, cbits, src, off);
    return group_list_radix_k<uint64_t>(h, pairs, n, cbits, src, off);
}

// Counting form of the grouping: per-target counts (warp-aggregated atomics
// over lanes with equal targets), their exclusive scan as the CSR offsets, an
// unordered scatter of the sources into a scratch array, then each target's
// sources written in ascending order by one warp: up to 32 by a bitonic
// network in registers, beyond that through a bitmap over the sources' index
// range in shared memory (the sources of one target are distinct cells), in
// windows of kSegBits indices.  The result equals the radix form's exactly; a
// repeated source (the traversal emits none) is detected and sends the list
// to the radix form, which keeps it.
constexpr int kSegWarps = 8;
constexpr int kSegWords = 1024;                  // bitmap words per warp
constexpr int kSegBits = 32 * kSegWords;         // source indices per window
constexpr int kSegPhys = kSegWords + kSegWords / 32;   // skewed: word j at j + j / 32

// With pcnt (the P2P list), also the particle-pair total sum n_T n_S.
__global__ void k_list_count(RegionList L, unsigned *cnt, const int *pcnt, unsigned long long *pairs_total)
{
    const int lane = (int)lane_id();
    unsigned long long np = 0;
    for_each_chunk(L, [&](int2 p, bool valid, int, unsigned) {
        const unsigned peers = __match_any_sync(kFull, p.x);
        if (p.x >= 0 && lane == __ffs(peers) - 1) atomicAdd(&cnt[p.x], (unsigned)__popc(peers));
        if (pcnt && valid) np += (unsigned long long)pcnt[p.x] * (unsigned long long)pcnt[p.y];
    });
    if (pcnt) {
        np = warp_sum(np);
        if (lane == 0 && np) atomicAdd(pairs_total, np);
    }
}

// tmp[off[t] + slot] = s for every pair (t, s); the slots of a target are
// handed out downwards from its count (cnt[] ends at zero).
__global__ void k_list_scatter(RegionList L, const unsigned *off, unsigned *cnt, int *tmp)
{
    const int lane = (int)lane_id();
    for_each_chunk(L, [&](int2 p, bool, int, unsigned) {
        const unsigned peers = __match_any_sync(kFull, p.x);
        const int leader = __ffs(peers) - 1;
        const unsigned k = (unsigned)__popc(peers);
        unsigned top = 0;
        if (p.x >= 0 && lane == leader) top = atomicSub(&cnt[p.x], k);
        top = __shfl_sync(kFull, top, leader);
        if (p.x >= 0) tmp[off[p.x] + top - k + __popc(peers & lanemask_lt())] = p.y;
    });
}

__device__ __forceinline__ int warp_sort32(int v, int lane)
{
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int o = __shfl_xor_sync(kFull, v, j);
            const bool up = (lane & k) == 0, lower = (lane & j) == 0;
            v = (lower == up) ? min(v, o) : max(v, o);
        }
    return v;
}

__global__ void __launch_bounds__(kSegWarps * 32) k_list_segsort(int nc, const unsigned *off, const int *tmp,
                                                                  int *src, unsigned *repeated, unsigned bit)
{
    __shared__ unsigned bitmap[kSegWarps][kSegPhys];
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= nc) return;
    const int lane = (int)lane_id();
    const unsigned b = off[t], L = off[t + 1] - b;
    if (L == 0) return;
    const int *si = tmp + b;
    int *so = src + b;
    if (L <= 32) {
        int v = lane < (int)L ? si[lane] : INT_MAX;
        v = warp_sort32(v, lane);
        if (lane < (int)L) so[lane] = v;
        return;
    }
    int lo = INT_MAX, hi = 0;
    for (unsigned i = lane; i < L; i += 32) {
        const int v = si[i];
        lo = min(lo, v);
        hi = max(hi, v);
    }
    lo = __reduce_min_sync(kFull, lo);
    hi = __reduce_max_sync(kFull, hi);
    unsigned *bm = bitmap[threadIdx.x >> 5];
    unsigned written = 0;
    for (int c0 = lo; c0 <= hi; c0 += kSegBits) {
        const int nw = min(kSegWords, (hi - c0) / 32 + 1);   // words of this window
        for (int j = lane; j < nw; j += 32) bm[j + (j >> 5)] = 0u;
        __syncwarp();
        for (unsigned i = lane; i < L; i += 32) {
            const int v = si[i] - c0;
            if (v >= 0 && v < 32 * nw) atomicOr(&bm[(v >> 5) + (v >> 10)], 1u << (v & 31));
        }
        __syncwarp();
        // lane l owns the words [l per, (l + 1) per): counts, their scan, then the indices in order
        const int per = (nw + 31) / 32;
        const int j0 = min(lane * per, nw), j1 = min(j0 + per, nw);
        unsigned c = 0;
        for (int j = j0; j < j1; ++j) c += __popc(bm[j + (j >> 5)]);
        unsigned incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned u = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += u;
        }
        unsigned pos = written + incl - c;
        for (int j = j0; j < j1; ++j) {
            unsigned x = bm[j + (j >> 5)];
            while (x) {
                so[pos++] = c0 + 32 * j + (__ffs(x) - 1);
                x &= x - 1u;
            }
        }
        written += __shfl_sync(kFull, incl, 31);
        __syncwarp();
    }
    if (written != L && lane == 0) atomicOr(repeated, bit);
}

// Group the (target, source) pairs by target into CSR form: off[c] .. off[c+1]
// are the sources of target c, ascending.  A repeated (target, source) pair
// sets `bit` in ctr->seg_long (read once the list is complete, which then
// regroups that list with the radix form).  Runs on `stream` with the given
// scratch (count / offset array, unordered sources, scan blocks).
static int group_list(Handle &h, cudaStream_t stream, DevBuf &lcnt, DevBuf &lkeys, DevBuf &scan_tmp,
                      const RegionList &L, int64_t n, DevBuf &src, DevBuf &off, unsigned bit,
                      const int *pcnt = nullptr, unsigned long long *pairs_total = nullptr)
{
    const int nc = (int)h.ncells;
    FMM_TRY(src.reserve(std::max<int64_t>(n, 1) * sizeof(int)));
    FMM_TRY(off.reserve((size_t)(nc + 1) * sizeof(int)));
    FMM_TRY(lcnt.reserve((size_t)(nc + 1) * sizeof(unsigned)));
    FMM_TRY(lkeys.reserve(std::max<int64_t>(n, 1) * sizeof(int)));
    unsigned *cnt = lcnt.as<unsigned>();
    unsigned *offu = reinterpret_cast<unsigned *>(off.as<int>());
    FMM_CUDA(cudaMemsetAsync(cnt, 0, (size_t)(nc + 1) * sizeof(unsigned), stream));
    const int gb = L.nreg;   // one block per region
    if (n > 0) {
        ++h.launches;
        k_list_count<<<gb, 256, 0, stream>>>(L, cnt, pcnt, pairs_total);
    }
    FMM_TRY(scan_exclusive_u32_on(h, stream, scan_tmp, cnt, offu, nc + 1, nullptr));
    if (n > 0) {
        ++h.launches;
        k_list_scatter<<<gb, 256, 0, stream>>>(L, offu, cnt, lkeys.as<int>());
        ++h.launches;
        k_list_segsort<<<ceil_div((int64_t)nc * 32, kSegWarps * 32), kSegWarps * 32, 0, stream>>>(
            nc, offu, lkeys.as<int>(), src.as<int>(), &h.counters.as<TravCounters>()->seg_long, bit);
    }
    FMM_CHECK_LAUNCH("group list");
    return FMM_OK;
}

// The M2L list is grouped on the handle's second stream (created on first
// use), beside the P2P list, the mutual split and the work items.
// join_lists_begin makes the handle's stream wait for it and copies its flag
// to the host; join_lists_end (after the stream is synchronised) regroups the
// list by radix sort if it repeats a pair.
static int side_stream(Handle &h)
{
    if (h.side) return FMM_OK;
    FMM_CUDA(cudaStreamCreateWithFlags(&h.side, cudaStreamNonBlocking));
    FMM_CUDA(cudaEventCreateWithFlags(&h.ev_fork, cudaEventDisableTiming));
    FMM_CUDA(cudaEventCreateWithFlags(&h.ev_join, cudaEventDisableTiming));
    return FMM_OK;
}

int join_lists_begin(Handle &h)
{
    if (!h.side_pending) return FMM_OK;
    FMM_CUDA(cudaStreamWaitEvent(h.stream, h.ev_join, 0));
    TravCounters *ctr = h.counters.as<TravCounters>();
    FMM_CUDA(cudaMemcpyAsync(&h.pinned->ctr.seg_long, &ctr->seg_long, sizeof(unsigned), cudaMemcpyDeviceToHost,
                             h.stream));
    return FMM_OK;
}

int join_lists_end(Handle &h)
{
    if (!h.side_pending) return FMM_OK;
    h.side_pending = false;
    if (h.pinned->ctr.seg_long & 1u) {
        const RegionList lm2l = {h.m2l_raw.as<int2>(), h.trav_reg.as<unsigned>(), (unsigned)h.m2l_cap,
                                 h.num_sms * kStackBlocksPerSM};
        FMM_TRY(group_list_radix(h, lm2l, h.n_m2l, h.m2l_src, h.m2l_off));
        FMM_CUDA(cudaStreamSynchronize(h.stream));
    }
    return FMM_OK;
}

int build_lists(Handle &h)
{
    const int nc = (int)h.ncells;
    if (nc >= (1 << 28)) {
        // the work stack packs a cell's first child into 28 bits
        set_error("dual tree traversal: more than 2^28 cells");
        return FMM_ERR_CAPACITY;
    }
    FMM_TRY(h.c_kids.reserve(nc * sizeof(int2)));
    ++h.launches;
    k_pack_kids<<<ceil_div(nc, 256), 256, 0, h.stream>>>(nc, h.c_cbeg.as<int>(), h.c_ccnt.as<int>(),
                                                         h.c_kids.as<int2>());
    FMM_TRY(h.counters.reserve(sizeof(TravCounters)));
    TravCounters *ctr = h.counters.as<TravCounters>();
    TravCounters *hc = &h.pinned->ctr;

    // leaf list (all leaves, in cell order)
    FMM_TRY(h.leaf_list.reserve(nc * sizeof(int)));
    FMM_CUDA(cudaMemsetAsync(ctr, 0, sizeof(TravCounters), h.stream));
    ++h.launches;
    k_leaf_list<<<ceil_div(nc, 256), 256, 0, h.stream>>>(nc, h.c_ccnt.as<int>(), h.leaf_list.as<int>(),
                                                         &ctr->nleaves);
    FMM_CHECK_LAUNCH("leaf list");

    phase_begin(h, FMM_PHASE_TRAVERSE);
    const int stack_blocks = h.num_sms * kStackBlocksPerSM;
    const int nreg = stack_blocks;   // one region per work-stack block
    auto round32 = [](int64_t v) { return (v + 31) / 32 * 32; };
    if (h.m2l_cap == 0) {
        h.m2l_cap = round32(((int64_t)nc * 64 + 1024) / nreg + 256);
        h.p2p_cap = round32(((int64_t)nc * 32 + 1024) / nreg + 256);
        h.front_cap = (int64_t)nc * 8 + 4096;
    }
    // seeding rounds: each splits one side of every frontier pair, so the frontier
    // grows by at most 8x per round; enough rounds for ~4 seeds per resident warp
    const int64_t seed_target = (int64_t)stack_blocks * kStackWarps * 4;
    int nrounds = 0;
    for (int64_t f = 1; f < seed_target && nrounds < 2 * h.nlevels && nrounds < 15; f *= 8) ++nrounds;
    const int round_blocks = h.num_sms * 16;
    FMM_TRY(h.trav_reg.reserve((size_t)2 * nreg * sizeof(unsigned)));
    unsigned *reg = h.trav_reg.as<unsigned>();
    for (int attempt = 0;; ++attempt) {
        FMM_TRY(h.m2l_raw.reserve((size_t)nreg * h.m2l_cap * sizeof(int2)));
        FMM_TRY(h.p2p_raw.reserve((size_t)nreg * h.p2p_cap * sizeof(int2)));
        FMM_TRY(h.front[0].reserve(h.front_cap * sizeof(int2)));
        FMM_TRY(h.front[1].reserve(h.front_cap * sizeof(int2)));
        // zero the counters, keeping the leaf count found above
        FMM_CUDA(cudaMemsetAsync(ctr, 0, offsetof(TravCounters, nleaves), h.stream));
        FMM_CUDA(cudaMemsetAsync(&ctr->round_count[0], 0, sizeof(ctr->round_count), h.stream));
        FMM_CUDA(cudaMemsetAsync(reg, 0, (size_t)2 * nreg * sizeof(unsigned), h.stream));
        TravArgs a;
        a.geom = h.c_geom.as<float4>();
        a.kids = h.c_kids.as<int2>();
        a.pcnt = h.c_pcnt.as<int>();
        a.theta = h.theta;
        a.hybrid_min = h.hybrid_min_pairs;
        a.m2l = h.m2l_raw.as<int2>();
        a.p2p = h.p2p_raw.as<int2>();
        a.cap_m2l = (unsigned)h.m2l_cap;
        a.cap_p2p = (unsigned)h.p2p_cap;
        a.reg = reg;
        a.nreg = nreg;
        a.next_cap = h.front_cap;
        a.n_next = nullptr;
        a.claim = nullptr;
        a.ctr = ctr;
        if (h.nlevels <= 1) {
            // the root is a leaf: the single P2P pair (root, root), region 0
            int2 rp = make_int2(0, 0);
            h.pinned->level_total = 1u;
            FMM_CUDA(cudaMemcpyAsync(h.p2p_raw.p, &rp, sizeof(int2), cudaMemcpyHostToDevice, h.stream));
            FMM_CUDA(cudaMemcpyAsync(reg + nreg, &h.pinned->level_total, sizeof(unsigned), cudaMemcpyHostToDevice,
                                     h.stream));
            FMM_CUDA(cudaStreamSynchronize(h.stream));
            h.n_m2l = 0;
            h.n_p2p = 1;
            break;
        }
        // the pair (root, root) is the frontier of seeding round 0
        h.pinned->ctr = TravCounters();
        h.pinned->ctr.round_count[0] = 1;
        int2 root = make_int2(0, 0);
        FMM_CUDA(cudaMemcpyAsync(h.front[0].p, &root, sizeof(int2), cudaMemcpyHostToDevice, h.stream));
        FMM_CUDA(cudaMemcpyAsync(&ctr->round_count[0], &h.pinned->ctr.round_count[0], sizeof(unsigned long long),
                                 cudaMemcpyHostToDevice, h.stream));
        // 1. seeding rounds, back to back
        int cur = 0;
        for (int r = 0; r < nrounds; ++r) {
            a.next = h.front[cur ^ 1].as<int2>();
            ++h.launches;
            k_dtt_round<<<round_blocks, 256, 0, h.stream>>>(h.front[cur].as<int2>(), &ctr->round_count[r],
                                                            &ctr->round_count[r + 1], a);
            cur ^= 1;
        }
        FMM_CHECK_LAUNCH("dtt rounds");
        // 2. work-stack passes on the last frontier: pass p claims the seeds counted
        //    in pass_count[p] and spills into pass_count[p + 1]; kPassesPerSync
        //    passes run back to back, then the host checks for spills left over
        bool overflow = false;
        const unsigned long long *nseeds_dev = &ctr->round_count[nrounds];
        for (int pass = 0;; pass += kPassesPerSync) {
            if (pass >= kMaxStackPasses) {
                set_error("dual tree traversal: work-stack pass limit reached");
                return FMM_ERR_CAPACITY;
            }
            // seeds first (on later passes they sit in pass_count[kPassesPerSync]), then reset the rest
            FMM_CUDA(cudaMemcpyAsync(&ctr->pass_count[0], nseeds_dev, sizeof(unsigned long long),
                                     cudaMemcpyDeviceToDevice, h.stream));
            FMM_CUDA(cudaMemsetAsync(&ctr->pass_claim[0], 0, sizeof(ctr->pass_claim), h.stream));
            FMM_CUDA(cudaMemsetAsync(&ctr->pass_count[1], 0, kPassesPerSync * sizeof(unsigned long long), h.stream));
            for (int p = 0; p < kPassesPerSync; ++p) {
                a.next = h.front[cur ^ 1].as<int2>();
                a.n_next = &ctr->pass_count[p + 1];
                a.claim = &ctr->pass_claim[p];
                ++h.launches;
                k_dtt_stack<<<stack_blocks, kStackWarps * 32, 0, h.stream>>>(h.front[cur].as<int2>(),
                                                                             &ctr->pass_count[p], a);
                cur ^= 1;
            }
            ++h.launches;
            k_region_totals<<<1, 256, 0, h.stream>>>(nreg, reg, ctr);
            FMM_CHECK_LAUNCH("dtt stack");
            FMM_CUDA(cudaMemcpyAsync(hc, ctr, sizeof(TravCounters), cudaMemcpyDeviceToHost, h.stream));
            FMM_CUDA(cudaStreamSynchronize(h.stream));
            if (hc->overflow) {
                overflow = true;
                break;
            }
            if (hc->pass_count[kPassesPerSync] == 0) break;
            nseeds_dev = &ctr->pass_count[kPassesPerSync];   // copied into pass_count[0] above
        }
        if (!overflow) {
            h.n_m2l = (int64_t)hc->n_m2l;
            h.n_p2p = (int64_t)hc->n_p2p;
            break;
        }
        if (attempt >= 12) {
            char msg[256];
            snprintf(msg, sizeof(msg),
                     "dual tree traversal: buffers still overflow after %d regrowths (flags %u, region caps m2l %lld "
                     "p2p %lld, frontier %lld)",
                     attempt, hc->overflow, (long long)h.m2l_cap, (long long)h.p2p_cap, (long long)h.front_cap);
            set_error(msg);
            return FMM_ERR_CAPACITY;
        }
        // The region counters keep counting past their capacity, so the largest
        // is the size needed (a lower bound if the traversal was cut short by a
        // frontier overflow): grow to 5/4 of it, at least double, and run again.
        unsigned long long max_round = 0;
        for (int r = 0; r <= nrounds; ++r) max_round = std::max(max_round, hc->round_count[r]);
        for (int p = 0; p <= kPassesPerSync; ++p) max_round = std::max(max_round, hc->pass_count[p]);
        if (hc->overflow & kOvM2L)
            h.m2l_cap = round32(std::max<int64_t>(h.m2l_cap * 2, (int64_t)hc->reg_max[0] * 5 / 4 + 256));
        if (hc->overflow & kOvP2P)
            h.p2p_cap = round32(std::max<int64_t>(h.p2p_cap * 2, (int64_t)hc->reg_max[1] * 5 / 4 + 256));
        if (hc->overflow & kOvNext) h.front_cap = std::max<int64_t>(h.front_cap * 2, (int64_t)(max_round * 3 / 2) + 4096);
        if (h.m2l_cap > 0x7fffffe0ll || h.p2p_cap > 0x7fffffe0ll) {
            set_error("dual tree traversal: list region capacity above 2^31");
            return FMM_ERR_CAPACITY;
        }
    }
    phase_end(h, FMM_PHASE_TRAVERSE);

    phase_begin(h, FMM_PHASE_LISTS);
    const RegionList lm2l = {h.m2l_raw.as<int2>(), reg, (unsigned)h.m2l_cap, nreg};
    const RegionList lp2p = {h.p2p_raw.as<int2>(), reg + nreg, (unsigned)h.p2p_cap, nreg};
    // the P2P particle-pair total (for the counters) comes with the P2P list's counts
    FMM_CUDA(cudaMemsetAsync(&ctr->p2p_pairs, 0, sizeof(unsigned long long), h.stream));
    FMM_TRY(side_stream(h));
    FMM_CUDA(cudaEventRecord(h.ev_fork, h.stream));
    FMM_CUDA(cudaStreamWaitEvent(h.side, h.ev_fork, 0));
    FMM_TRY(group_list(h, h.side, h.lcnt_side, h.lkeys_side, h.scan_tmp_side, lm2l, h.n_m2l, h.m2l_src, h.m2l_off,
                       1u));
    FMM_CUDA(cudaEventRecord(h.ev_join, h.side));
    h.side_pending = true;
    FMM_TRY(group_list(h, h.stream, h.lcnt, h.lkeys, h.scan_tmp, lp2p, h.n_p2p, h.p2p_src, h.p2p_off, 2u,
                       h.c_pcnt.as<int>(), &ctr->p2p_pairs));
    FMM_CUDA(cudaMemcpyAsync(hc, ctr, sizeof(TravCounters), cudaMemcpyDeviceToHost, h.stream));
    FMM_CUDA(cudaStreamSynchronize(h.stream));
    h.p2p_pairs = (int64_t)hc->p2p_pairs;
    h.nleaves = hc->nleaves;
    // a repeated (target, source) pair in the P2P list: regroup it by radix sort
    // (the M2L list's flag is read when its stream is joined)
    if (hc->seg_long & 2u) FMM_TRY(group_list_radix(h, lp2p, h.n_p2p, h.p2p_src, h.p2p_off));
    phase_end(h, FMM_PHASE_LISTS);
    return FMM_OK;
}

}  // namespace fmm
