// p2p.cu -- near field: P2P over the P2P list, fused with L2P and the output scatter.
//
// P2P (Sec. 3.3, Table 4): phi_i += sum_j q_j / r_ij, grad_i += sum_j q_j (x_j - x_i) / r_ij^3
// over the particles j of every source leaf listed for the target leaf of i
// (pairs at distance 0 contribute nothing).  The paper's kernel is AVX with
// rsqrt_ps (Sec. 3.3); here:
//   - work item = (target leaf, slice of <= 16 of its targets); one warp per item;
//   - the 16 target positions sit in registers (warp-uniform); the listed
//     source leaves are merged into runs of consecutive siblings (one
//     contiguous block of particles in one frame), and the runs are staged
//     per warp in shared memory, 256 particles per chunk, double-buffered
//     with cp.async so the next chunk streams in while the current one is
//     used; each lane takes one staged source per step and computes its 16
//     pair interactions, two targets per packed FP32 instruction (FFMA2,
//     FADD2, FMUL2) and one SFU rsqrt per pair (13 FP32 operations, 6.5 issue
//     slots, 1 SFU operation per pair);
//   - positions are FP32 offsets from the centre of the leaf's parent (the
//     frame); a source is moved into the target's frame by the exact (dyadic)
//     shift X_frame(S) - X_frame(T), so close pairs keep ~2^-24 of the frame
//     size in absolute precision;
//   - the 4 x 16 accumulators are reduce-scattered across the warp (62
//     shuffles), then lanes 2g / 2g+1 own target g: L2P of the leaf's local
//     expansion is added, units restored (phi / h, grad / h^2) and the result
//     written at the caller's index.
// With FMM_FLAG_KAHAN each lane keeps its per-target sums as (sum, compensation)
// pairs, updated once per staged chunk (plain FP32 over the lane's 8 sources of
// the chunk, then one compensated add); work items then hold at most 8 targets
// so that the three accumulator sets stay in registers.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "fmm_internal.cuh"
#include "mi.cuh"
#include "p2p_common.cuh"

namespace fmm {

#ifndef FMM_P2P_G
#define FMM_P2P_G 16
#endif
constexpr int kP2PG = FMM_P2P_G;   // targets per work item (multiple of 4, at most 16)
constexpr int kP2PGKahan = 8;      // targets per work item with compensated accumulation
constexpr int kP2PThreads = 64;   // two warps per block: a block's slot is freed as soon as its two items end

#ifndef FMM_P2P_SLOTS
#define FMM_P2P_SLOTS 256
#endif
#ifndef FMM_P2P_MIN_BLOCKS
#define FMM_P2P_MIN_BLOCKS 6
#endif
#ifndef FMM_P2P_UNROLL
#define FMM_P2P_UNROLL 1
#endif
constexpr int kSlots = FMM_P2P_SLOTS;   // staged source particles per buffer
constexpr int kP2PUnroll = FMM_P2P_UNROLL;   // staged sources per lane per loop iteration
// Staging by bulk copies (cp.async.bulk, the TMA engine, completion on an
// mbarrier with bounded waits) instead of per-lane 16-byte cp.async: correct,
// but 3.5 % slower on this ALU-bound kernel (7.34 vs 7.08 ms at N = 1M, P = 8):
// one lane issues the copies and every lane polls the mbarrier.  Off by default.
#ifndef FMM_P2P_BULK
#define FMM_P2P_BULK 0
#endif
constexpr bool kP2PBulk = FMM_P2P_BULK != 0;
// 2 buffers x (particles + shifts) per warp, then two mbarriers per warp
constexpr int kP2PSmem = (kP2PThreads / 32) * (4 * kSlots * (int)sizeof(float4) + 2 * 8);


// Work items: one per slice of <= 16 targets of a leaf, slices balanced in size;
// item = (leaf cell, first target, target count, index of the leaf in the leaf list).
__global__ void k_p2p_item_count(int nleaves, const int *leaf_list, const int *pcnt, int g, unsigned *cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nleaves) return;
    const int nt = pcnt[leaf_list[i]];
    cnt[i] = (unsigned)((nt + g - 1) / g);
}

__global__ void k_p2p_item_write(int nleaves, const int *leaf_list, const int *pbeg, const int *pcnt, int g,
                                 const unsigned *off, int4 *items)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nleaves) return;
    const int c = leaf_list[i];
    const int nt = pcnt[c], b = pbeg[c];
    const int ns = (nt + g - 1) / g;
    for (int k = 0; k < ns; ++k) {
        const int t0 = (int)((int64_t)nt * k / ns), t1 = (int)((int64_t)nt * (k + 1) / ns);
        items[off[i] + k] = make_int4(c, b + t0, t1 - t0, i);
    }
}

// Source runs: maximal stretches of consecutive list entries whose leaves share
// a frame cell and follow each other in particle order (runs of siblings), so
// that a run is one contiguous block of particles in one frame.
__device__ __forceinline__ bool run_continues(int a, int b, const int *parent, const int *pbeg, const int *pcnt)
{
    return frame_of(parent, a) == frame_of(parent, b) && pbeg[a] + pcnt[a] == pbeg[b];
}

__global__ void k_p2p_run_count(int nleaves, const int *leaf_list, const int *off, const int *src, const int *parent,
                                const int *pbeg, const int *pcnt, unsigned *nruns)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nleaves) return;
    const int t = leaf_list[w];
    const int eb = off[t], ee = off[t + 1];
    unsigned n = 0;
    for (int e0 = eb; e0 < ee; e0 += 32) {
        const int e = e0 + (int)lane_id();
        bool start = false;
        if (e < ee) start = e == eb || !run_continues(src[e - 1], src[e], parent, pbeg, pcnt);
        n += __popc(__ballot_sync(kFull, start));
    }
    if (lane_id() == 0) nruns[w] = n;
}

// Run records: (X_frame(S) - X_frame(T), first particle) and the end particle.
__global__ void k_p2p_runs(int nleaves, const int *leaf_list, const int *off, const int *src, const int *parent,
                           const int *pbeg, const int *pcnt, const float4 *geom, const unsigned *roff, float4 *run,
                           int *run_end)
{
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nleaves) return;
    const unsigned lane = lane_id();
    const int t = leaf_list[w];
    const float4 Xt = geom[frame_of(parent, t)];
    const int eb = off[t], ee = off[t + 1];
    unsigned before = roff[w];
    for (int e0 = eb; e0 < ee; e0 += 32) {
        const int e = e0 + (int)lane;
        bool start = false, last = false;
        int s = 0;
        if (e < ee) {
            s = src[e];
            start = e == eb || !run_continues(src[e - 1], s, parent, pbeg, pcnt);
            last = e + 1 == ee || !run_continues(s, src[e + 1], parent, pbeg, pcnt);
        }
        const unsigned m = __ballot_sync(kFull, start);
        const unsigned r = before + __popc(m & (lanemask_lt() | (1u << lane))) - 1u;
        if (start) {
            const float4 Xs = geom[frame_of(parent, s)];
            run[r] = make_float4(Xs.x - Xt.x, Xs.y - Xt.y, Xs.z - Xt.z, __int_as_float(pbeg[s]));
        }
        if (last) run_end[r] = pbeg[s] + pcnt[s];
        before += __popc(m);
    }
}

// Accumulate the interactions of one source s (already in the target frame) with
// NT targets, two targets per packed FP32 instruction (FFMA2 / FADD2 / FMUL2):
// targets are held negated as float2 pairs (ntx[h] = -(t_2h, t_2h+1)), and
// acc[4h + k] is component k (potential, gradient x, y, z) of that pair.
// r^2 is accumulated on top of eps = FLT_MIN, which keeps rsqrt finite and
// leaves every squared distance representable in FP32 unchanged (only pairs
// that round to the same FP32 point see it).  kExact (chunks holding the target
// leaf's own particles): a pair at distance 0 (a particle meeting itself, or a
// coincident one) has r^2 = eps and contributes exactly nothing.
template <int NT, bool kExact>
__device__ __forceinline__ void p2p_tile(const float4 &s, const float2 *ntx, const float2 *nty, const float2 *ntz,
                                         float2 *acc)
{
    constexpr float kEps = 1.17549435e-38f;
    constexpr int HG = 2;   // target pairs whose chains are written side by side (each step of both, then the next)
    const float2 sx = make_float2(s.x, s.x), sy = make_float2(s.y, s.y), sz = make_float2(s.z, s.z);
    const float2 sq = make_float2(s.w, s.w);
    const float2 eps = make_float2(kEps, kEps);
#pragma unroll
    for (int h0 = 0; h0 < NT / 2; h0 += HG) {
        float2 dx[HG], dy[HG], dz[HG], r2[HG], rinv[HG], qr[HG], qr3[HG];
#pragma unroll
        for (int j = 0; j < HG; ++j)
            if (h0 + j < NT / 2) {
                dx[j] = __fadd2_rn(sx, ntx[h0 + j]);
                dy[j] = __fadd2_rn(sy, nty[h0 + j]);
                dz[j] = __fadd2_rn(sz, ntz[h0 + j]);
            }
#pragma unroll
        for (int j = 0; j < HG; ++j)
            if (h0 + j < NT / 2) r2[j] = __ffma2_rn(dx[j], dx[j], eps);
#pragma unroll
        for (int j = 0; j < HG; ++j)
            if (h0 + j < NT / 2) r2[j] = __ffma2_rn(dy[j], dy[j], r2[j]);
#pragma unroll
        for (int j = 0; j < HG; ++j)
            if (h0 + j < NT / 2) r2[j] = __ffma2_rn(dz[j], dz[j], r2[j]);
#pragma unroll
        for (int j = 0; j < HG; ++j)
            if (h0 + j < NT / 2) {
                if (kExact) {
                    rinv[j].x = r2[j].x > kEps ? rsqrt_approx(r2[j].x) : 0.0f;
                    rinv[j].y = r2[j].y > kEps ? rsqrt_approx(r2[j].y) : 0.0f;
                } else {
                    rinv[j].x = rsqrt_approx(r2[j].x);
                    rinv[j].y = rsqrt_approx(r2[j].y);
                }
            }
#pragma unroll
        for (int j = 0; j < HG; ++j)
            if (h0 + j < NT / 2) {
                qr[j] = __fmul2_rn(sq, rinv[j]);
                qr3[j] = __fmul2_rn(qr[j], __fmul2_rn(rinv[j], rinv[j]));
            }
#pragma unroll
        for (int j = 0; j < HG; ++j)
            if (h0 + j < NT / 2) {
                const int h = h0 + j;
                acc[4 * h + 0] = __fadd2_rn(acc[4 * h + 0], qr[j]);
                acc[4 * h + 1] = __ffma2_rn(qr3[j], dx[j], acc[4 * h + 1]);
                acc[4 * h + 2] = __ffma2_rn(qr3[j], dy[j], acc[4 * h + 2]);
                acc[4 * h + 3] = __ffma2_rn(qr3[j], dz[j], acc[4 * h + 3]);
            }
    }
}

// The source stream of one work item: double-buffered staging (the next chunk is
// copied while the current one is used) and NT targets per staged source.
// With kKahan the per-chunk partial sums (blk) are added to v with Kahan
// compensation (comp) once per chunk.
// Returns false if a bulk-copy wait gave up (the item's results are then not
// written; the caller flags the error).
template <int NT, bool kKahan>
__device__ __forceinline__ bool p2p_stream(RunCursor &cur, const float4 *run, const int *run_end, const float4 *pos,
                                           float4 *buf, unsigned long long *mbar, int lb0, int lb1,
                                           const float2 *ntx, const float2 *nty, const float2 *ntz, float2 *v,
                                           float2 *comp, float2 *blk)
{
    const int lane = (int)lane_id();
    bool self_cur = false, self_next = false;
    int n_cur;
    if (kP2PBulk) {
        n_cur = cur.stage_bulk<kSlots>(run, run_end, pos, buf, buf + kSlots, lb0, lb1, &self_cur, mbar);
    } else {
        n_cur = cur.stage<kSlots, false>(run, run_end, pos, nullptr, buf, nullptr, buf + kSlots, lb0, lb1,
                                         &self_cur);
        cp_async_commit();
    }
    for (int c = 0; n_cur > 0; ++c) {
        float4 *cur_part = buf + (c & 1) * (2 * kSlots);
        float4 *cur_shift = cur_part + kSlots;
        float4 *nx = buf + ((c + 1) & 1) * (2 * kSlots);
        int n_next;
        if (kP2PBulk) {
            // buffer b's j-th fill completes phase j of mbar[b]: chunk c is fill c / 2 of buffer c & 1
            n_next = cur.stage_bulk<kSlots>(run, run_end, pos, nx, nx + kSlots, lb0, lb1, &self_next,
                                            mbar + ((c + 1) & 1));
            if (!mbar_wait_warp(mbar + (c & 1), (unsigned)(c >> 1) & 1u)) {
                // give up on this item, but let the copies already issued land first
                mbar_wait_warp(mbar + ((c + 1) & 1), (unsigned)((c + 1) >> 1) & 1u);
                return false;
            }
        } else {
            n_next = cur.stage<kSlots, false>(run, run_end, pos, nullptr, nx, nullptr, nx + kSlots, lb0, lb1,
                                              &self_next);
            cp_async_commit();
            cp_async_wait_1();
        }
        __syncwarp();
        float2 *acc = kKahan ? blk : v;
#pragma unroll kP2PUnroll
        for (int t0 = 0; t0 < n_cur; t0 += 32) {
            const int j = t0 + lane;
            float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < n_cur) {
                s = cur_part[j];
                const float4 d = cur_shift[j];
                s.x += d.x;
                s.y += d.y;
                s.z += d.z;
            }
            if (self_cur) p2p_tile<NT, true>(s, ntx, nty, ntz, acc);
            else p2p_tile<NT, false>(s, ntx, nty, ntz, acc);
        }
        if (kKahan) {
#pragma unroll
            for (int i = 0; i < 2 * NT; ++i) {
                const float2 y = make_float2(blk[i].x - comp[i].x, blk[i].y - comp[i].y);
                const float2 t = make_float2(v[i].x + y.x, v[i].y + y.y);
                comp[i] = make_float2((t.x - v[i].x) - y.x, (t.y - v[i].y) - y.y);
                v[i] = t;
                blk[i] = make_float2(0.0f, 0.0f);
            }
        }
        __syncwarp();   // every lane is done with this buffer before it is refilled
        n_cur = n_next;
        self_cur = self_next;
    }
    return true;
}

template <int P, bool kKahan, int G>
__global__ void __launch_bounds__(kP2PThreads, FMM_P2P_MIN_BLOCKS) k_p2p(int nitems, const int4 *items, const unsigned *roff,
                                                     const float4 *run, const int *run_end, const float4 *racc,
                                                     const float4 *pos, const int *pbeg, const int *pcnt, const int *level,
                                                     const int *parent, const float4 *geom, const float *L,
                                                     const int *perm, float phi_scale, float grad_scale,
                                                     const float2 *cell_scale, float *phi, float *grad,
                                                     float *phi_sorted, unsigned *err)
{
    static_assert(G % 4 == 0 && G <= 16, "targets per item");
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    extern __shared__ float4 p2p_smem[];
    const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= nitems) return;
    const unsigned lane = lane_id();
    float4 *buf = p2p_smem + (threadIdx.x >> 5) * (4 * kSlots);   // [2][particles, shifts][kSlots]
    unsigned long long *mbar = reinterpret_cast<unsigned long long *>(p2p_smem + (kP2PThreads / 32) * (4 * kSlots)) +
                               2 * (threadIdx.x >> 5);
    if (kP2PBulk) {
        if (lane == 0) {
            mbar_init(mbar, 1);
            mbar_init(mbar + 1, 1);
            fence_mbar_init();
        }
        __syncwarp();
    }
    const int4 it = items[item];
    const int leaf = it.x, tb = it.y, tc = it.z;
    const int lb0 = pbeg[leaf], lb1 = lb0 + pcnt[leaf];   // the target leaf's own particles

    // targets (offsets from the target frame centre, warp-uniform), negated, in
    // float2 pairs; extra slots repeat the last target
    float2 ntx[G / 2], nty[G / 2], ntz[G / 2];
#pragma unroll
    for (int h = 0; h < G / 2; ++h) {
        const float4 p0 = pos[tb + min(2 * h, tc - 1)];
        const float4 p1 = pos[tb + min(2 * h + 1, tc - 1)];
        ntx[h] = make_float2(-p0.x, -p1.x);
        nty[h] = make_float2(-p0.y, -p1.y);
        ntz[h] = make_float2(-p0.z, -p1.z);
    }
    // a[4 h + k]: component k (potential, gradient x, y, z) of targets 2h, 2h+1
    float2 a[2 * G];
#pragma unroll
    for (int i = 0; i < 2 * G; ++i) a[i] = make_float2(0.0f, 0.0f);
    float2 comp[kKahan ? 2 * G : 1];
    float2 blk[kKahan ? 2 * G : 1];
    if (kKahan) {
#pragma unroll
        for (int i = 0; i < 2 * G; ++i) comp[i] = blk[i] = make_float2(0.0f, 0.0f);
    }

    RunCursor cur;
    cur.init(roff, it.w, run, run_end);
    // the item computes tc rounded up to 4 (tc <= 8) or to 2 (tc > 8) targets, extra
    // ones repeating the last target: balanced slices of leaves of 13-55
    // particles hold 9-16 targets, where rounding to 4 would add ~9 % of pairs
    const int ntr = tc <= 4 ? 4 : tc <= 8 ? 8 : (tc + 1) & ~1;
    bool staged = true;
    if (ntr == 4) {
        staged = p2p_stream<4, kKahan>(cur, run, run_end, pos, buf, mbar, lb0, lb1, ntx, nty, ntz, a, comp, blk);
    } else if (G <= 8 || ntr == 8) {
        staged = p2p_stream<(G < 8 ? G : 8), kKahan>(cur, run, run_end, pos, buf, mbar, lb0, lb1, ntx, nty, ntz, a, comp, blk);
    } else if (ntr == 10) {
        staged = p2p_stream<(G < 10 ? G : 10), kKahan>(cur, run, run_end, pos, buf, mbar, lb0, lb1, ntx, nty, ntz, a, comp, blk);
    } else if (ntr == 12) {
        staged = p2p_stream<(G < 12 ? G : 12), kKahan>(cur, run, run_end, pos, buf, mbar, lb0, lb1, ntx, nty, ntz, a, comp, blk);
    } else if (ntr == 14) {
        staged = p2p_stream<(G < 14 ? G : 14), kKahan>(cur, run, run_end, pos, buf, mbar, lb0, lb1, ntx, nty, ntz, a, comp, blk);
    } else {
        staged = p2p_stream<G, kKahan>(cur, run, run_end, pos, buf, mbar, lb0, lb1, ntx, nty, ntz, a, comp, blk);
    }
    if (!staged) {   // a bulk-copy wait gave up: flag it, write nothing for this item
        if (lane == 0) atomicOr(err, 2u);
        return;
    }
    if (kKahan) {   // fold the outstanding compensation into the sums
#pragma unroll
        for (int i = 0; i < 2 * G; ++i) a[i] = make_float2(a[i].x - comp[i].x, a[i].y - comp[i].y);
    }
    // v[4 g + k]: component k of target g (zero-padded to 16 targets)
    float v[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) v[i] = 0.0f;
#pragma unroll
    for (int h = 0; h < G / 2; ++h)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[4 * (2 * h) + k] = a[4 * h + k].x;
            v[4 * (2 * h + 1) + k] = a[4 * h + k].y;
        }

    warp_reduce_scatter64(v);
    // lane 2g holds (phi, gx) of target g, lane 2g+1 holds (gy, gz)
    const float o0 = __shfl_down_sync(kFull, v[0], 1);
    const float o1 = __shfl_down_sync(kFull, v[1], 1);
    const int g = (int)(lane >> 1);
    if ((lane & 1u) || g >= tc) return;
    const int sidx = tb + g;
    const float4 p = pos[sidx];
    float pot = v[0], gx = v[1], gy = o0, gz = o1;
    if (racc) {   // the mutual pass's sums for this target
        const float4 r = racc[sidx];
        pot += r.x;
        gx += r.y;
        gy += r.z;
        gz += r.w;
    }

    // L2P: phi += sum_n Lb_n w_n(r / s), grad += (1/s) sum_m Lb_{m + e_d} w_m(r / s),
    // r = u - X_leaf = d - (X_leaf - X_frame)
    {
        const float inv_s = ldexpf(1.0f, level[leaf]);
        const float4 Xc = geom[leaf], Xf = geom[frame_of(parent, leaf)];
        float w[T];
        taylor_monomials<P>(fmaf(p.x, inv_s, -(Xc.x - Xf.x) * inv_s), fmaf(p.y, inv_s, -(Xc.y - Xf.y) * inv_s),
                            fmaf(p.z, inv_s, -(Xc.z - Xf.z) * inv_s), w);
        const float *Lc = L + (size_t)leaf * TP;
        float lp = 0.0f, lx = 0.0f, ly = 0.0f, lz = 0.0f;
#pragma unroll
        for (int nm = 0; nm < P; ++nm)
#pragma unroll
            for (int a = nm; a >= 0; --a)
#pragma unroll
                for (int b = nm - a; b >= 0; --b) {
                    const int c = nm - a - b;
                    const float wm = w[MI<P>::idx(a, b, c)];
                    lp = fmaf(Lc[MI<P>::idx(a, b, c)], wm, lp);
                    if (nm + 1 < P) {
                        lx = fmaf(Lc[MI<P>::idx(a + 1, b, c)], wm, lx);
                        ly = fmaf(Lc[MI<P>::idx(a, b + 1, c)], wm, ly);
                        lz = fmaf(Lc[MI<P>::idx(a, b, c + 1)], wm, lz);
                    }
                }
        pot += lp;
        gx = fmaf(lx, inv_s, gx);
        gy = fmaf(ly, inv_s, gy);
        gz = fmaf(lz, inv_s, gz);
    }
    if (cell_scale) {   // cells of several systems: each leaf carries its system's units
        const float2 cs = cell_scale[leaf];
        phi_scale = cs.x;
        grad_scale = cs.y;
    }
    const int dst = perm[sidx];
    const float ph = pot * phi_scale;
    if (phi) phi[dst] = ph;
    if (phi_sorted) phi_sorted[sidx] = ph;
    if (grad) {
        grad[3 * (int64_t)dst + 0] = gx * grad_scale;
        grad[3 * (int64_t)dst + 1] = gy * grad_scale;
        grad[3 * (int64_t)dst + 2] = gz * grad_scale;
    }
}

// Work items of at most g targets over the leaf list (g = targets per warp item).
int build_work_items(Handle &h, int g, DevBuf &items, int64_t &n_items)
{
    const int nl = (int)h.nleaves;
    FMM_TRY(h.c_tmp.reserve((size_t)(2 * nl + 1) * sizeof(unsigned)));
    unsigned *cnt = h.c_tmp.as<unsigned>(), *off = cnt + nl, *tot = off + nl;
    ++h.launches;
    k_p2p_item_count<<<ceil_div(nl, 256), 256, 0, h.stream>>>(nl, h.leaf_list.as<int>(), h.c_pcnt.as<int>(), g, cnt);
    FMM_TRY(scan_exclusive_u32(h, cnt, off, nl, tot));
    FMM_CUDA(cudaMemcpyAsync(&h.pinned->level_total, tot, sizeof(unsigned), cudaMemcpyDeviceToHost, h.stream));
    FMM_CUDA(cudaStreamSynchronize(h.stream));
    n_items = h.pinned->level_total;
    FMM_TRY(items.reserve(std::max<int64_t>(n_items, 1) * sizeof(int4)));
    ++h.launches;
    k_p2p_item_write<<<ceil_div(nl, 256), 256, 0, h.stream>>>(nl, h.leaf_list.as<int>(), h.c_pbeg.as<int>(),
                                                              h.c_pcnt.as<int>(), g, off, items.as<int4>());
    FMM_CHECK_LAUNCH("p2p items");
    return FMM_OK;
}

// Source runs of the lists (off, src) of every leaf: run offsets per leaf-list
// entry (roff, nleaves + 1), run records and end particles.  The buffers are
// sized for max_runs (a run starts at a list entry, so the list's length
// bounds it) without reading the count back; with nruns the count is read
// back too (one host round trip).
int build_runs(Handle &h, const int *off, const int *src, int64_t max_runs, DevBuf &roff_buf, DevBuf &ent,
               DevBuf &cnt, int64_t *nruns)
{
    const int nl = (int)h.nleaves;
    FMM_TRY(h.c_tmp.reserve((size_t)(nl + 1) * sizeof(unsigned)));
    unsigned *nrun = h.c_tmp.as<unsigned>();
    FMM_TRY(roff_buf.reserve((size_t)(nl + 1) * sizeof(unsigned)));
    unsigned *roff = roff_buf.as<unsigned>();
    ++h.launches;
    k_p2p_run_count<<<ceil_div((int64_t)nl * 32, 256), 256, 0, h.stream>>>(
        nl, h.leaf_list.as<int>(), off, src, h.c_parent.as<int>(), h.c_pbeg.as<int>(), h.c_pcnt.as<int>(), nrun);
    FMM_TRY(scan_exclusive_u32(h, nrun, roff, nl, roff + nl));
    FMM_TRY(ent.reserve(std::max<int64_t>(max_runs, 1) * sizeof(float4)));
    FMM_TRY(cnt.reserve(std::max<int64_t>(max_runs, 1) * sizeof(int)));
    ++h.launches;
    k_p2p_runs<<<ceil_div((int64_t)nl * 32, 256), 256, 0, h.stream>>>(
        nl, h.leaf_list.as<int>(), off, src, h.c_parent.as<int>(), h.c_pbeg.as<int>(), h.c_pcnt.as<int>(),
        h.c_geom.as<float4>(), roff, ent.as<float4>(), cnt.as<int>());
    FMM_CHECK_LAUNCH("p2p runs");
    if (nruns) {
        FMM_CUDA(cudaMemcpyAsync(&h.pinned->level_total, roff + nl, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                 h.stream));
        FMM_CUDA(cudaStreamSynchronize(h.stream));
        *nruns = h.pinned->level_total;
    }
    return FMM_OK;
}

// The runs of the full lists (one-sided near field, adjoint, batched forms);
// with the mutual schedule they are built on first use.
int ensure_full_runs(Handle &h)
{
    if (h.full_runs_ready) return FMM_OK;
    FMM_TRY(build_runs(h, h.p2p_off.as<int>(), h.p2p_src.as<int>(), h.n_p2p, h.p2p_poff, h.p2p_ent, h.p2p_cnt,
                       &h.n_pieces));
    h.full_runs_ready = true;
    return FMM_OK;
}

int build_p2p_items(Handle &h)
{
    // the mutual schedule's split of the lists, or the source runs of every
    // target leaf's whole list
    h.mutual_ready = false;
    h.full_runs_ready = false;
    if (h.flags & FMM_FLAG_MUTUAL) FMM_TRY(build_mutual(h));
    else FMM_TRY(ensure_full_runs(h));
    // work items (the adjoint's items are built on first use)
    h.adj_items_ready = false;
    h.tc_items_ready = false;
    h.p2p_g = 0;
    return build_work_items(h, (h.flags & FMM_FLAG_KAHAN) ? kP2PGKahan : kP2PG, h.p2p_items, h.n_items);
}

template <int P, bool kKahan, int G> static int p2p_launch(Handle &h, float *phi, float *grad)
{
    static bool configured[64] = {};
    if (h.device >= 0 && h.device < 64 && !configured[h.device]) {
        FMM_CUDA(cudaFuncSetAttribute(k_p2p<P, kKahan, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, kP2PSmem));
        configured[h.device] = true;
    }
    const float phi_scale = (float)(1.0 / h.norm_host[3]);
    const float grad_scale = (float)(1.0 / (h.norm_host[3] * h.norm_host[3]));
    const int blocks = ceil_div((int64_t)h.n_items * 32, kP2PThreads);
    ++h.launches;
    // with the mutual schedule this pass covers the one-sided entries and adds
    // the accumulated mutual sums
    const bool mu = h.mutual_ready;
    k_p2p<P, kKahan, G><<<blocks, kP2PThreads, kP2PSmem, h.stream>>>(
        (int)h.n_items, h.p2p_items.as<int4>(), (mu ? h.os_poff : h.p2p_poff).as<unsigned>(),
        (mu ? h.os_ent : h.p2p_ent).as<float4>(), (mu ? h.os_cnt : h.p2p_cnt).as<int>(),
        mu ? h.racc.as<float4>() : nullptr, h.pos.as<float4>(), h.c_pbeg.as<int>(), h.c_pcnt.as<int>(), h.c_level.as<int>(),
        h.c_parent.as<int>(), h.c_geom.as<float4>(), h.L.as<float>(), h.perm.as<int>(), phi_scale, grad_scale,
        h.c_scale.as<float2>(), phi, grad, h.phi_sorted.as<float>(), h.err_flag.as<unsigned>());
    FMM_CHECK_LAUNCH("p2p");
    return FMM_OK;
}

// The work items must have been built with the matching target count
// (kP2PGKahan with FMM_FLAG_KAHAN, else h.p2p_g or kP2PG).
template <int P> static int p2p_impl(Handle &h, float *phi, float *grad)
{
    if (h.flags & FMM_FLAG_KAHAN) return p2p_launch<P, true, kP2PGKahan>(h, phi, grad);
    if (h.p2p_g == 8) return p2p_launch<P, false, 8>(h, phi, grad);
    return p2p_launch<P, false, kP2PG>(h, phi, grad);
}

int evaluate_p2p(Handle &h, float *phi, float *grad)
{
    FMM_TRY(h.phi_sorted.reserve(h.N * sizeof(float)));
    if (h.mutual_ready) FMM_TRY(p2p_mutual(h));
    switch (h.P) {
    case 3: return p2p_impl<3>(h, phi, grad);
    case 4: return p2p_impl<4>(h, phi, grad);
    case 5: return p2p_impl<5>(h, phi, grad);
    case 6: return p2p_impl<6>(h, phi, grad);
    case 8: return p2p_impl<8>(h, phi, grad);
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED;
    }
}

// ---------------------------------------------------------------------------
// energy E = 1/2 sum_i q_i phi_i, reduced in FP64
// ---------------------------------------------------------------------------
constexpr int kEnergyThreads = 256;

__global__ void __launch_bounds__(kEnergyThreads) k_energy_partial(int64_t n, const float4 *pos, const float *phi,
                                                                   double *part)
{
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)pos[i].w * (double)phi[i];
    s = warp_sum(s);
    __shared__ double ws[kEnergyThreads / 32];
    if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kEnergyThreads / 32; ++k) t += ws[k];
        part[blockIdx.x] = t;
    }
}

__global__ void k_energy_final(int nb, const double *part, double *E)
{
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[b];
    s = warp_sum(s);
    __shared__ double ws[32];
    if (lane_id() == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += ws[k];
        *E = 0.5 * t;
    }
}

int energy_reduce(Handle &h, double *E)
{
    const int nb = std::min(ceil_div(h.N, kEnergyThreads), h.num_sms * 4);
    FMM_TRY(h.energy_part.reserve((size_t)(nb + 1) * sizeof(double)));
    double *part = h.energy_part.as<double>();
    ++h.launches;
    k_energy_partial<<<nb, kEnergyThreads, 0, h.stream>>>(h.N, h.pos.as<float4>(), h.phi_sorted.as<float>(), part);
    ++h.launches;
    k_energy_final<<<1, 256, 0, h.stream>>>(nb, part, part + nb);
    FMM_CHECK_LAUNCH("energy");
    FMM_CUDA(cudaMemcpyAsync(E, part + nb, sizeof(double), cudaMemcpyDeviceToHost, h.stream));
    FMM_CUDA(cudaStreamSynchronize(h.stream));
    return FMM_OK;
}

}  // namespace fmm
