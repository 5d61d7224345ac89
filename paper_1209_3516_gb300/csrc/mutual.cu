// mutual.cu -- mutual (Newton's third law) near field: each unordered leaf pair once.
//
// The paper's method descends from falcON (Sec. 2), whose near field evaluates
// every pair of leaves once and applies the interaction to both of them.  The
// P2P lists that Algorithm 4 emits here are symmetric in practice ((A, B) is
// listed iff (B, A) is; the split rule can break this when two cells have
// equal radii, so every mirror is checked), and with FMM_FLAG_MUTUAL each
// target leaf's list is split into
//   - its mutual part: sources B > A whose mirror entry (B, A) exists, and
//   - its one-sided part: B == A, and any entry without a mirror (checked by
//     a binary search for A in B's sorted list from the entry with B > A; none
//     are expected).
// The mutual pass takes, for every work item of A's targets and every source
// particle s of its mutual runs, both directions of each pair term:
//   phi_t += q_s / r,  grad_t += q_s (u_s - u_t) / r^3   (target side, registers)
//   phi_s += q_t / r,  grad_s += q_t (u_t - u_s) / r^3   (reaction: the lane
//                                                         holding s, over the item's targets)
// and adds both into an accumulator in sorted order with vector float
// reductions (red.global.add.v4.f32 / .v2.f32): the reaction once per (item,
// source particle), the target side once per (item, target).  The ordinary P2P
// kernel then runs over the one-sided runs and adds the accumulator before the
// L2P and the scatter to caller order.  A pair term costs 18 packed FP32
// instructions per four interactions (two targets, both directions) instead
// of 13 per two, and one SFU rsqrt per two interactions.  The order of the
// floating-point reductions is not fixed, so results are reproducible to
// rounding, not bitwise.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "fmm_internal.cuh"
#include "p2p_common.cuh"

namespace fmm {

// ---------------------------------------------------------------------------
// list split
// ---------------------------------------------------------------------------
// Entry kinds (one byte per list entry, preset to 2): 0 skip (the mirror's
// mutual entry covers it), 1 mutual, 2 one-sided.  One warp per leaf A; each
// entry B > A looks A up in B's sorted list by binary search: found, the entry
// is mutual and its mirror is skipped; not found, both stay one-sided.
// Entries B == A, and B < A whose mirror was not found, stay one-sided.  Each
// lane runs the searches of two entries (e and e + 32) in lockstep, so that
// their dependent loads overlap.
__global__ void k_mutual_mark(int nleaves, const int *leaf_list, const int *off, const int *src, unsigned char *kind)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nleaves) return;
    const int t = leaf_list[w];
    const int eb = off[t], ee = off[t + 1];
    for (int e = eb + (int)lane_id(); e < ee; e += 64) {
        const int e2 = e + 32;
        const int b1 = src[e], b2 = e2 < ee ? src[e2] : -1;
        // [lo, hi) search ranges; an empty range for an entry that does not search
        int lo1 = 0, hi1 = 0, lo2 = 0, hi2 = 0;
        if (b1 > t) {
            lo1 = off[b1];
            hi1 = off[b1 + 1];
        }
        if (b2 > t) {
            lo2 = off[b2];
            hi2 = off[b2 + 1];
        }
        int m1 = -1, m2 = -1;
        while (lo1 < hi1 || lo2 < hi2) {
            const int c1 = (lo1 + hi1) >> 1, c2 = (lo2 + hi2) >> 1;
            const int v1 = lo1 < hi1 ? src[c1] : 0, v2 = lo2 < hi2 ? src[c2] : 0;
            if (lo1 < hi1) {
                if (v1 == t) {
                    m1 = c1;
                    hi1 = lo1;
                } else if (v1 < t) lo1 = c1 + 1;
                else hi1 = c1;
            }
            if (lo2 < hi2) {
                if (v2 == t) {
                    m2 = c2;
                    hi2 = lo2;
                } else if (v2 < t) lo2 = c2 + 1;
                else hi2 = c2;
            }
        }
        if (m1 >= 0) {
            kind[e] = 1;
            kind[m1] = 0;
        }
        if (m2 >= 0) {
            kind[e2] = 1;
            kind[m2] = 0;
        }
    }
}

// One warp per leaf: its counts of mutual and one-sided entries.
__global__ void k_mutual_count(int nleaves, const int *leaf_list, const int *off, const unsigned char *kind,
                               unsigned *cnt_mu, unsigned *cnt_os)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nleaves) return;
    const int t = leaf_list[w];
    const int eb = off[t], ee = off[t + 1];
    unsigned nm = 0, no = 0;
    for (int e0 = eb; e0 < ee; e0 += 32) {
        const int e = e0 + (int)lane_id();
        const int k = e < ee ? kind[e] : 0;
        nm += __popc(__ballot_sync(kFull, k == 1));
        no += __popc(__ballot_sync(kFull, k == 2));
    }
    if (lane_id() == 0) {
        cnt_mu[t] = nm;
        cnt_os[t] = no;
    }
}

// One warp per leaf: its entries into the two lists, in list (source) order.
__global__ void k_mutual_write(int nleaves, const int *leaf_list, const int *off, const int *src,
                               const unsigned char *kind, const unsigned *mu_off, const unsigned *os_off, int *mu_src,
                               int *os_src)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nleaves) return;
    const unsigned lane = lane_id();
    const int t = leaf_list[w];
    const int eb = off[t], ee = off[t + 1];
    unsigned pm = mu_off[t], po = os_off[t];
    for (int e0 = eb; e0 < ee; e0 += 32) {
        const int e = e0 + (int)lane;
        const int s = e < ee ? src[e] : 0;
        const int k = e < ee ? kind[e] : 0;
        const unsigned bm = __ballot_sync(kFull, k == 1), bo = __ballot_sync(kFull, k == 2);
        if (k == 1) mu_src[pm + __popc(bm & lanemask_lt())] = s;
        if (k == 2) os_src[po + __popc(bo & lanemask_lt())] = s;
        pm += __popc(bm);
        po += __popc(bo);
    }
}

// Split the grouped P2P lists and build the source runs of both parts.
int build_mutual(Handle &h)
{
    const int nl = (int)h.nleaves;
    const int64_t nc = h.ncells;
    FMM_TRY(h.mu_off.reserve((size_t)(nc + 1) * sizeof(unsigned)));
    FMM_TRY(h.os_off.reserve((size_t)(nc + 1) * sizeof(unsigned)));
    FMM_TRY(h.mu_cnt_tmp.reserve((size_t)(2 * nc) * sizeof(unsigned) + (size_t)std::max<int64_t>(h.n_p2p, 1)));
    unsigned *cm = h.mu_cnt_tmp.as<unsigned>(), *co = cm + nc;
    unsigned char *kind = reinterpret_cast<unsigned char *>(co + nc);   // one byte per list entry
    FMM_CUDA(cudaMemsetAsync(cm, 0, (size_t)(2 * nc) * sizeof(unsigned), h.stream));
    FMM_CUDA(cudaMemsetAsync(kind, 2, (size_t)std::max<int64_t>(h.n_p2p, 1), h.stream));
    const int blocks = ceil_div((int64_t)nl * 32, 256);
    ++h.launches;
    k_mutual_mark<<<blocks, 256, 0, h.stream>>>(nl, h.leaf_list.as<int>(), h.p2p_off.as<int>(), h.p2p_src.as<int>(),
                                                kind);
    ++h.launches;
    k_mutual_count<<<blocks, 256, 0, h.stream>>>(nl, h.leaf_list.as<int>(), h.p2p_off.as<int>(), kind, cm, co);
    unsigned *mo = h.mu_off.as<unsigned>(), *oo = h.os_off.as<unsigned>();
    FMM_TRY(scan_exclusive_u32(h, cm, mo, nc, mo + nc));
    FMM_TRY(scan_exclusive_u32(h, co, oo, nc, oo + nc));
    // both parts are sized for the whole list (no count read back)
    FMM_TRY(h.mu_src.reserve(std::max<int64_t>(h.n_p2p, 1) * sizeof(int)));
    FMM_TRY(h.os_src.reserve(std::max<int64_t>(h.n_p2p, 1) * sizeof(int)));
    ++h.launches;
    k_mutual_write<<<blocks, 256, 0, h.stream>>>(nl, h.leaf_list.as<int>(), h.p2p_off.as<int>(), h.p2p_src.as<int>(),
                                                 kind, mo, oo, h.mu_src.as<int>(), h.os_src.as<int>());
    FMM_CHECK_LAUNCH("mutual list split");
    FMM_TRY(build_runs(h, h.mu_off.as<int>(), h.mu_src.as<int>(), h.n_p2p, h.mu_poff, h.mu_ent, h.mu_cnt, nullptr));
    FMM_TRY(build_runs(h, h.os_off.as<int>(), h.os_src.as<int>(), h.n_p2p, h.os_poff, h.os_ent, h.os_cnt, nullptr));
    FMM_TRY(h.racc.reserve((size_t)h.N * sizeof(float4)));
    h.mutual_ready = true;
    return FMM_OK;
}

// ---------------------------------------------------------------------------
// mutual P2P pass
// ---------------------------------------------------------------------------
constexpr int kMuG = 16;           // targets per work item (the P2P items)
constexpr int kMuThreads = 64;     // two warps per block
#ifndef FMM_MU_SLOTS
#define FMM_MU_SLOTS 256
#endif
constexpr int kMuSlots = FMM_MU_SLOTS;   // staged sources per buffer
constexpr int kMuSmem = (kMuThreads / 32) * (4 * kMuSlots + kMuG) * (int)sizeof(float4);
#ifndef FMM_MU_PER_LANE
#define FMM_MU_PER_LANE 2
#endif
constexpr int kMuPerLane = FMM_MU_PER_LANE;   // staged sources per lane per step (the default shape)
// The second shape the many-systems autotuner tries: 4 staged sources per
// lane at 4 blocks per SM.
constexpr int kMuPerLaneWide = 4, kMuMinBlocksWide = 4;
#ifndef FMM_MU_MIN_BLOCKS
#define FMM_MU_MIN_BLOCKS 6
#endif
#ifndef FMM_MU_TARGETS_SMEM
#define FMM_MU_TARGETS_SMEM 1
#endif
// 1: the item's targets sit in shared memory (read by broadcast), so that the
// kernel fits 168 registers and 6 blocks (12 warps) per SM; 0: in registers
// (244 registers, 4 blocks per SM).  N = 1M, P = 8, theta = 0.5, mutual pass:
// registers / 4 blocks / 4 sources per lane 5.03 ms; shared / 6 / 2: 4.74 ms;
// shared / 6 / 3 (166 registers) 5.14; shared / 7-8 blocks with 192 staged
// sources per buffer (spills) 5.00-5.08.
constexpr bool kMuTargetsSmem = FMM_MU_TARGETS_SMEM != 0;
constexpr int kMuTargetF4 = kMuG;   // per warp: (ntx, nty) and (ntz, nqt) float4 of each target pair

__device__ __forceinline__ void red_add_v4(float4 *addr, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}
__device__ __forceinline__ void red_add_v2(float *addr, float a, float b)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(addr), "f"(a), "f"(b) : "memory");
}

// Stage up to kMuSlots sources of the item's runs: positions (with charges) by
// cp.async, the frame shift with the particle's index (as int bits in w).
__device__ __forceinline__ int mu_stage(RunCursor &cur, const float4 *run, const int *run_end, const float4 *pos,
                                        float4 *part, float4 *shift)
{
    const int lane = (int)lane_id();
    int slots = 0;
    while (slots < kMuSlots && cur.e < cur.e1) {
        const int m = min(cur.cnt - cur.o, kMuSlots - slots);
        const int begin = cur.pb + cur.o;
        for (int i = lane; i < m; i += 32) {
            cp_async16(part + slots + i, pos + begin + i);
            shift[slots + i] = make_float4(cur.shx, cur.shy, cur.shz, __int_as_float(begin + i));
        }
        slots += m;
        cur.o += m;
        if (cur.o == cur.cnt) {
            ++cur.e;
            cur.o = 0;
            cur.load(run, run_end);
        }
    }
    return slots;
}

// Both directions of the pair terms of U sources (in the target frame, charges
// in w) with NT targets, two per packed instruction: ntx.. negated target
// positions, nqt negated target charges; acc[4h + k] the target side, ps, gs
// the sources' reactions (ps accumulates -phi_s).
// Pair bodies whose stages are written side by side (each stage of all of
// them, then the next); N = 1M, mutual pass: 1 / 2 / 4 / 8 bodies 4.73-4.75 /
// 4.74 / 4.71 / 4.91 ms.
#ifndef FMM_MU_SIDE
#define FMM_MU_SIDE 4
#endif
constexpr int kMuSide = FMM_MU_SIDE;

template <int NT, int U>
__device__ __forceinline__ void mu_tile(const float4 *s, const float2 *ntx_r, const float2 *nty_r,
                                        const float2 *ntz_r, const float2 *nqt_r, const float4 *tsm, float2 *acc,
                                        float2 *ps, float2 *gsx, float2 *gsy, float2 *gsz)
{
    constexpr float kEps = 1.17549435e-38f;
    constexpr int NB = (NT / 2) * U;   // bodies (target pair h, source u), body i = h U + u
    constexpr int B = kMuSide;
    const float2 eps = make_float2(kEps, kEps);
#pragma unroll
    for (int i0 = 0; i0 < NB; i0 += B) {
        float2 tx[B], ty[B], tz[B], tq[B], dx[B], dy[B], dz[B], r2[B], rinv[B], rinv3[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int i = i0 + j;
            if (i >= NB) continue;
            const int h = i / U, u = i % U;
            if constexpr (kMuTargetsSmem) {
                const float4 a = tsm[2 * h], b = tsm[2 * h + 1];
                tx[j] = make_float2(a.x, a.y);
                ty[j] = make_float2(a.z, a.w);
                tz[j] = make_float2(b.x, b.y);
                tq[j] = make_float2(b.z, b.w);
            } else {
                tx[j] = ntx_r[h];
                ty[j] = nty_r[h];
                tz[j] = ntz_r[h];
                tq[j] = nqt_r[h];
            }
            dx[j] = __fadd2_rn(make_float2(s[u].x, s[u].x), tx[j]);
            dy[j] = __fadd2_rn(make_float2(s[u].y, s[u].y), ty[j]);
            dz[j] = __fadd2_rn(make_float2(s[u].z, s[u].z), tz[j]);
        }
#pragma unroll
        for (int j = 0; j < B; ++j)
            if (i0 + j < NB) r2[j] = __ffma2_rn(dx[j], dx[j], eps);
#pragma unroll
        for (int j = 0; j < B; ++j)
            if (i0 + j < NB) r2[j] = __ffma2_rn(dy[j], dy[j], r2[j]);
#pragma unroll
        for (int j = 0; j < B; ++j)
            if (i0 + j < NB) r2[j] = __ffma2_rn(dz[j], dz[j], r2[j]);
#pragma unroll
        for (int j = 0; j < B; ++j)
            if (i0 + j < NB) rinv[j] = make_float2(rsqrt_approx(r2[j].x), rsqrt_approx(r2[j].y));
#pragma unroll
        for (int j = 0; j < B; ++j)
            if (i0 + j < NB) rinv3[j] = __fmul2_rn(__fmul2_rn(rinv[j], rinv[j]), rinv[j]);
#pragma unroll
        for (int j = 0; j < B; ++j) {
            const int i = i0 + j;
            if (i >= NB) continue;
            const int h = i / U, u = i % U;
            const float2 sq = make_float2(s[u].w, s[u].w);
            // target side: phi_t += q_s / r, grad_t += q_s e / r^3
            acc[4 * h + 0] = __ffma2_rn(sq, rinv[j], acc[4 * h + 0]);
            const float2 qs3 = __fmul2_rn(sq, rinv3[j]);
            acc[4 * h + 1] = __ffma2_rn(qs3, dx[j], acc[4 * h + 1]);
            acc[4 * h + 2] = __ffma2_rn(qs3, dy[j], acc[4 * h + 2]);
            acc[4 * h + 3] = __ffma2_rn(qs3, dz[j], acc[4 * h + 3]);
            // reaction: -phi_s += (-q_t) / r, grad_s += (-q_t) e / r^3
            ps[u] = __ffma2_rn(tq[j], rinv[j], ps[u]);
            const float2 qt3 = __fmul2_rn(tq[j], rinv3[j]);
            gsx[u] = __ffma2_rn(qt3, dx[j], gsx[u]);
            gsy[u] = __ffma2_rn(qt3, dy[j], gsy[u]);
            gsz[u] = __ffma2_rn(qt3, dz[j], gsz[u]);
        }
    }
}

template <int NT, int U>
__device__ __forceinline__ void mu_stream(RunCursor &cur, const float4 *run, const int *run_end, const float4 *pos,
                                          float4 *buf, const float2 *ntx, const float2 *nty, const float2 *ntz,
                                          const float2 *nqt, const float4 *tsm, float2 *acc, float4 *racc)
{
    const int lane = (int)lane_id();
    int n_cur = mu_stage(cur, run, run_end, pos, buf, buf + kMuSlots);
    cp_async_commit();
    for (int c = 0; n_cur > 0; ++c) {
        float4 *cur_part = buf + (c & 1) * (2 * kMuSlots);
        float4 *cur_shift = cur_part + kMuSlots;
        float4 *nx = buf + ((c + 1) & 1) * (2 * kMuSlots);
        const int n_next = mu_stage(cur, run, run_end, pos, nx, nx + kMuSlots);
        cp_async_commit();
        cp_async_wait_1();
        __syncwarp();
#pragma unroll 1
        for (int t0 = 0; t0 < n_cur; t0 += 32 * U) {
            // U staged sources per lane per step: independent chains side by side
            float4 s[U];
            int sidx[U];
            float2 ps[U], gsx[U], gsy[U], gsz[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = t0 + 32 * u + lane;
                s[u] = make_float4(1e20f, 1e20f, 1e20f, 0.f);   // past the count: far away, no charge
                sidx[u] = -1;
                if (j < n_cur) {
                    s[u] = cur_part[j];
                    const float4 d = cur_shift[j];
                    s[u].x += d.x;
                    s[u].y += d.y;
                    s[u].z += d.z;
                    sidx[u] = __float_as_int(d.w);
                }
                ps[u] = gsx[u] = gsy[u] = gsz[u] = make_float2(0.f, 0.f);
            }
            mu_tile<NT, U>(s, ntx, nty, ntz, nqt, tsm, acc, ps, gsx, gsy, gsz);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (sidx[u] >= 0)
                    red_add_v4(racc + sidx[u], -(ps[u].x + ps[u].y), gsx[u].x + gsx[u].y, gsy[u].x + gsy[u].y,
                               gsz[u].x + gsz[u].y);
        }
        __syncwarp();   // every lane is done with this buffer before it is refilled
        n_cur = n_next;
    }
}

// One warp per work item (<= 16 targets of a leaf) over its mutual runs, U
// staged sources per lane per step.
template <int U, int MinBlocks>
__global__ void __launch_bounds__(kMuThreads, MinBlocks)
    k_p2p_mutual(int nitems, const int4 *items, const unsigned *roff, const float4 *run, const int *run_end,
                 const float4 *pos, float4 *racc)
{
    extern __shared__ float4 mu_smem[];
    const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= nitems) return;
    const unsigned lane = lane_id();
    float4 *buf = mu_smem + (threadIdx.x >> 5) * (4 * kMuSlots + kMuG);
    float4 *tsm = buf + 4 * kMuSlots;   // the targets (shared-memory form)
    const int4 it = items[item];
    const int tb = it.y, tc = it.z;
    RunCursor cur;
    cur.init(roff, it.w, run, run_end);
    if (cur.e >= cur.e1) return;   // no mutual sources
    // targets (negated positions and charges, float2 pairs); slots past the
    // count repeat the last target's position with charge 0 (no reaction)
    float2 ntx[kMuTargetsSmem ? 1 : kMuG / 2], nty[kMuTargetsSmem ? 1 : kMuG / 2],
        ntz[kMuTargetsSmem ? 1 : kMuG / 2], nqt[kMuTargetsSmem ? 1 : kMuG / 2];
    if constexpr (kMuTargetsSmem) {
        if (lane < (unsigned)(kMuG / 2)) {
            const int h = (int)lane;
            const float4 p0 = pos[tb + min(2 * h, tc - 1)];
            const float4 p1 = pos[tb + min(2 * h + 1, tc - 1)];
            tsm[2 * h] = make_float4(-p0.x, -p1.x, -p0.y, -p1.y);
            tsm[2 * h + 1] = make_float4(-p0.z, -p1.z, 2 * h < tc ? -p0.w : 0.0f, 2 * h + 1 < tc ? -p1.w : 0.0f);
        }
        __syncwarp();
    } else {
#pragma unroll
        for (int h = 0; h < kMuG / 2; ++h) {
            const float4 p0 = pos[tb + min(2 * h, tc - 1)];
            const float4 p1 = pos[tb + min(2 * h + 1, tc - 1)];
            ntx[h] = make_float2(-p0.x, -p1.x);
            nty[h] = make_float2(-p0.y, -p1.y);
            ntz[h] = make_float2(-p0.z, -p1.z);
            nqt[h] = make_float2(2 * h < tc ? -p0.w : 0.0f, 2 * h + 1 < tc ? -p1.w : 0.0f);
        }
    }
    float2 a[2 * kMuG];
#pragma unroll
    for (int i = 0; i < 2 * kMuG; ++i) a[i] = make_float2(0.0f, 0.0f);
    const int ntr = tc <= 4 ? 4 : tc <= 8 ? 8 : tc <= 12 ? 12 : 16;
    if (ntr == 4) mu_stream<4, U>(cur, run, run_end, pos, buf, ntx, nty, ntz, nqt, tsm, a, racc);
    else if (ntr == 8) mu_stream<8, U>(cur, run, run_end, pos, buf, ntx, nty, ntz, nqt, tsm, a, racc);
    else if (ntr == 12) mu_stream<12, U>(cur, run, run_end, pos, buf, ntx, nty, ntz, nqt, tsm, a, racc);
    else mu_stream<16, U>(cur, run, run_end, pos, buf, ntx, nty, ntz, nqt, tsm, a, racc);
    // target side: reduce-scatter, lanes 2g / 2g + 1 add (phi, gx) / (gy, gz) of target g
    float v[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = 0.0f;
#pragma unroll
    for (int h = 0; h < kMuG / 2; ++h)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[4 * (2 * h) + k] = a[4 * h + k].x;
            v[4 * (2 * h + 1) + k] = a[4 * h + k].y;
        }
    warp_reduce_scatter64(v);
    const int g = (int)(lane >> 1);
    if (g < tc) red_add_v2(reinterpret_cast<float *>(racc + tb + g) + 2 * (lane & 1u), v[0], v[1]);
}

template <int U, int MinBlocks> static int p2p_mutual_launch(Handle &h)
{
    static bool configured[64] = {};
    if (h.device >= 0 && h.device < 64 && !configured[h.device]) {
        FMM_CUDA(cudaFuncSetAttribute(k_p2p_mutual<U, MinBlocks>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      kMuSmem));
        configured[h.device] = true;
    }
    FMM_CUDA(cudaMemsetAsync(h.racc.p, 0, (size_t)h.N * sizeof(float4), h.stream));
    ++h.launches;
    k_p2p_mutual<U, MinBlocks><<<ceil_div((int64_t)h.n_items * 32, kMuThreads), kMuThreads, kMuSmem, h.stream>>>(
        (int)h.n_items, h.p2p_items.as<int4>(), h.mu_poff.as<unsigned>(), h.mu_ent.as<float4>(), h.mu_cnt.as<int>(),
        h.pos.as<float4>(), h.racc.as<float4>());
    FMM_CHECK_LAUNCH("mutual p2p");
    return FMM_OK;
}

int p2p_mutual(Handle &h)
{
    if (h.mu_lanes == kMuPerLaneWide) return p2p_mutual_launch<kMuPerLaneWide, kMuMinBlocksWide>(h);
    return p2p_mutual_launch<kMuPerLane, FMM_MU_MIN_BLOCKS>(h);
}

}  // namespace fmm
