// adjoint.cu -- near field of fmm_backward: the adjoint P2P over the P2P list,
// fused with the L2P terms of both far fields and the scatter to caller order.
//
// The paper has no adjoint; these are the derivatives of the sums of Sec. 3.2.
// For upstream gradients a_i = dL/dphi_i and b_i = dL/dgrad_i (b' = b / h in
// normalised coordinates) and the charges q of the last evaluation,
//   dq_k = Psi(u_k),   dx_k = a_k grad(u_k) + H(u_k) b'_k + q_k grad Psi(u_k)
// (then / h and / h^2 for physical units), where Psi is the field of charges a
// and dipoles b' and grad, H are the gradient and Hessian of the potential of
// q.  Far field: Psi comes from the adjoint expansions La (dipole P2M, then the
// same M2M, M2L, L2L as the forward pass), grad and H from the forward local
// expansions L.  Near field: for a target t and a source s at offset
// e = u_s - u_t, r = |e|, the three terms of one pair combine into
//   dq_t += a_s / r - (b'_s . e) / r^3
//   dx_t += [ C + (S - 3 (C . e) / r^2) e ] / r^3,
//   S = q_t a_s + a_t q_s,   C = q_t b'_s - q_s b'_t,
// so each target keeps four accumulators, as in the forward P2P.
//
// Layout: one warp per work item of <= 8 targets of a leaf; targets
// (position in the frame of the leaf's parent, q, a, b') sit in registers;
// the item's source runs are staged per warp in shared memory (positions,
// adjoint sources and frame shifts; 128 particles per chunk, double-buffered
// with cp.async); each lane takes one staged source and computes its pairs
// with every target (two targets per packed FP32 instruction: 16 issue slots
// and one SFU rsqrt per pair).  The
// 4 x 8 sums are reduce-scattered so that lane 4g + k owns component k of
// target g, which then adds its far-field terms and writes the result.
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "fmm_internal.cuh"
#include "mi.cuh"
#include "p2p_common.cuh"

namespace fmm {

constexpr int kAdjG = 8;          // targets per work item
constexpr int kAdjThreads = 128;
constexpr int kAdjSlots = 128;    // staged sources per buffer
constexpr int kAdjSmem = (kAdjThreads / 32) * 2 * 3 * kAdjSlots * (int)sizeof(float4);   // 48 KiB

// Per-target operands of the pair terms, two targets per float2 (packed FP32):
// negated positions, q, a and negated b'.
struct AdjTargets {
    float2 nx[4], ny[4], nz[4], q[4], a[4], nbx[4], nby[4], nbz[4];
};

__device__ __forceinline__ float2 bcast(float v) { return make_float2(v, v); }

// Pairs of one source (sp = position in the target frame and q, sa = (a, b'))
// with NT targets, two per packed FP32 instruction (FFMA2 / FADD2 / FMUL2):
// 32 packed operations and two SFU rsqrt per two pairs.  acc[4 h + k] holds
// component k (dq, dx, dy, dz) of targets 2h, 2h+1.
template <int NT, bool kExact>
__device__ __forceinline__ void adj_tile(const float4 &sp, const float4 &sa, const AdjTargets &t, float2 *acc)
{
    constexpr float kEps = 1.17549435e-38f;   // FLT_MIN: keeps rsqrt finite, see the forward P2P
    const float2 eps = bcast(kEps), m3 = bcast(-3.0f);
    const float2 sx = bcast(sp.x), sy = bcast(sp.y), sz = bcast(sp.z), sq = bcast(sp.w);
    const float2 sa2 = bcast(sa.x), sbx = bcast(sa.y), sby = bcast(sa.z), sbz = bcast(sa.w);
    const float2 nsbx = bcast(-sa.y), nsby = bcast(-sa.z), nsbz = bcast(-sa.w);
#pragma unroll
    for (int h = 0; h < NT / 2; ++h) {
        const float2 ex = __fadd2_rn(sx, t.nx[h]), ey = __fadd2_rn(sy, t.ny[h]), ez = __fadd2_rn(sz, t.nz[h]);
        const float2 r2 = __ffma2_rn(ez, ez, __ffma2_rn(ey, ey, __ffma2_rn(ex, ex, eps)));
        float2 rinv;
        if (kExact) {
            rinv.x = r2.x > kEps ? rsqrt_approx(r2.x) : 0.0f;
            rinv.y = r2.y > kEps ? rsqrt_approx(r2.y) : 0.0f;
        } else {
            rinv.x = rsqrt_approx(r2.x);
            rinv.y = rsqrt_approx(r2.y);
        }
        const float2 rinv2 = __fmul2_rn(rinv, rinv);
        const float2 rinv3 = __fmul2_rn(rinv2, rinv);
        // dq: a_s / r - (b'_s . e) / r^3
        const float2 nbse = __ffma2_rn(nsbz, ez, __ffma2_rn(nsby, ey, __fmul2_rn(nsbx, ex)));
        acc[4 * h] = __ffma2_rn(nbse, rinv3, __ffma2_rn(sa2, rinv, acc[4 * h]));
        // dx: [C + (S - 3 (C . e) / r^2) e] / r^3
        const float2 S = __ffma2_rn(t.q[h], sa2, __fmul2_rn(t.a[h], sq));
        const float2 cx = __ffma2_rn(t.q[h], sbx, __fmul2_rn(sq, t.nbx[h]));
        const float2 cy = __ffma2_rn(t.q[h], sby, __fmul2_rn(sq, t.nby[h]));
        const float2 cz = __ffma2_rn(t.q[h], sbz, __fmul2_rn(sq, t.nbz[h]));
        const float2 ce = __ffma2_rn(cz, ez, __ffma2_rn(cy, ey, __fmul2_rn(cx, ex)));
        const float2 f = __ffma2_rn(ce, __fmul2_rn(rinv2, m3), S);
        acc[4 * h + 1] = __ffma2_rn(__ffma2_rn(f, ex, cx), rinv3, acc[4 * h + 1]);
        acc[4 * h + 2] = __ffma2_rn(__ffma2_rn(f, ey, cy), rinv3, acc[4 * h + 2]);
        acc[4 * h + 3] = __ffma2_rn(__ffma2_rn(f, ez, cz), rinv3, acc[4 * h + 3]);
    }
}

template <int NT>
__device__ __forceinline__ void adj_stream(RunCursor &cur, const float4 *run, const int *run_end, const float4 *pos,
                                           const float4 *adj, float4 *buf, int lb0, int lb1, const AdjTargets &t,
                                           float2 *acc)
{
    const int lane = (int)lane_id();
    // buffer b: [pos | adj | shift] x kAdjSlots at buf + b * 3 * kAdjSlots
    bool self_cur = false, self_next = false;
    int n_cur = cur.stage<kAdjSlots, true>(run, run_end, pos, adj, buf, buf + kAdjSlots, buf + 2 * kAdjSlots, lb0,
                                           lb1, &self_cur);
    cp_async_commit();
    for (int c = 0; n_cur > 0; ++c) {
        const float4 *cp = buf + (c & 1) * (3 * kAdjSlots);
        float4 *nx = buf + ((c + 1) & 1) * (3 * kAdjSlots);
        const int n_next = cur.stage<kAdjSlots, true>(run, run_end, pos, adj, nx, nx + kAdjSlots, nx + 2 * kAdjSlots,
                                                      lb0, lb1, &self_next);
        cp_async_commit();
        cp_async_wait_1();
        __syncwarp();
        for (int t0 = 0; t0 < n_cur; t0 += 32) {
            const int j = t0 + lane;
            // padding lanes: a zero source far away (r^2 overflows to inf, 1/r to 0),
            // so that every term is an exact 0 (a zero source at the origin could
            // meet a target at the frame centre and give 0 * inf)
            float4 sp = make_float4(1e20f, 1e20f, 1e20f, 0.f), sa = make_float4(0.f, 0.f, 0.f, 0.f);
            if (j < n_cur) {
                sp = cp[j];
                sa = cp[kAdjSlots + j];
                const float4 d = cp[2 * kAdjSlots + j];
                sp.x += d.x;
                sp.y += d.y;
                sp.z += d.z;
            }
            if (self_cur) adj_tile<NT, true>(sp, sa, t, acc);
            else adj_tile<NT, false>(sp, sa, t, acc);
        }
        __syncwarp();   // every lane is done with this buffer before it is refilled
        n_cur = n_next;
        self_cur = self_next;
    }
}

// Reduce-scatter 32 values across the warp by recursive halving: lane l ends
// with the warp-wide sum of entry l in v[0].
__device__ __forceinline__ void warp_reduce_scatter32(float *v)
{
    const unsigned lane = lane_id();
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        const int half = 16 >> step;
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

template <int P>
__global__ void __launch_bounds__(kAdjThreads, 3)
    k_p2p_adj(int nitems, const int4 *items, const unsigned *roff, const float4 *run, const int *run_end,
              const float4 *pos, const float4 *adj, const int *pbeg, const int *pcnt, const int *level,
              const int *parent, const float4 *geom, const float *L, const float *La, const int *perm,
              float dq_scale, float dx_scale, float *dq, float *dx)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    extern __shared__ float4 adj_smem[];
    const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= nitems) return;
    const unsigned lane = lane_id();
    float4 *buf = adj_smem + (threadIdx.x >> 5) * (2 * 3 * kAdjSlots);
    const int4 it = items[item];
    const int leaf = it.x, tb = it.y, tc = it.z;
    const int lb0 = pbeg[leaf], lb1 = lb0 + pcnt[leaf];

    AdjTargets t;   // extra slots repeat the last target
#pragma unroll
    for (int h = 0; h < kAdjG / 2; ++h) {
        const int g0 = tb + min(2 * h, tc - 1), g1 = tb + min(2 * h + 1, tc - 1);
        const float4 p0 = pos[g0], p1 = pos[g1], b0 = adj[g0], b1 = adj[g1];
        t.nx[h] = make_float2(-p0.x, -p1.x);
        t.ny[h] = make_float2(-p0.y, -p1.y);
        t.nz[h] = make_float2(-p0.z, -p1.z);
        t.q[h] = make_float2(p0.w, p1.w);
        t.a[h] = make_float2(b0.x, b1.x);
        t.nbx[h] = make_float2(-b0.y, -b1.y);
        t.nby[h] = make_float2(-b0.z, -b1.z);
        t.nbz[h] = make_float2(-b0.w, -b1.w);
    }
    float2 a2[2 * kAdjG];
#pragma unroll
    for (int i = 0; i < 2 * kAdjG; ++i) a2[i] = make_float2(0.0f, 0.0f);
    RunCursor cur;
    cur.init(roff, it.w, run, run_end);
    if (tc <= 4) adj_stream<4>(cur, run, run_end, pos, adj, buf, lb0, lb1, t, a2);
    else if (tc <= 6) adj_stream<6>(cur, run, run_end, pos, adj, buf, lb0, lb1, t, a2);
    else adj_stream<kAdjG>(cur, run, run_end, pos, adj, buf, lb0, lb1, t, a2);
    // acc[4 g + k]: component k of target g
    float acc[4 * kAdjG];
#pragma unroll
    for (int h = 0; h < kAdjG / 2; ++h)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc[4 * (2 * h) + k] = a2[4 * h + k].x;
            acc[4 * (2 * h + 1) + k] = a2[4 * h + k].y;
        }

    warp_reduce_scatter32(acc);
    const int g = (int)(lane >> 2), k = (int)(lane & 3u);
    if (g >= tc) return;
    const int sidx = tb + g;
    const float4 p = pos[sidx], ab = adj[sidx];
    float v = acc[0];

    // far field at the target: r = u - X_leaf = d - (X_leaf - X_frame), scaled by 1/s
    const float inv_s = ldexpf(1.0f, level[leaf]);
    const float4 Xc = geom[leaf], Xf = geom[frame_of(parent, leaf)];
    float w[T];
    taylor_monomials<P>(fmaf(p.x, inv_s, -(Xc.x - Xf.x) * inv_s), fmaf(p.y, inv_s, -(Xc.y - Xf.y) * inv_s),
                        fmaf(p.z, inv_s, -(Xc.z - Xf.z) * inv_s), w);
    const float *Lq = L + (size_t)leaf * TP;
    const float *Lp = La + (size_t)leaf * TP;
    if (k == 0) {
        // Psi = sum_n La_n w_n
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < T; ++i) s = fmaf(Lp[i], w[i], s);
        v += s;
        if (dq) dq[perm[sidx]] = v * dq_scale;
        return;
    }
    // component c of a grad + H b' + q grad Psi:
    //   grad_c   = (1/s)   sum_m L_{m + e_c} w_m
    //   (H b')_c = (1/s^2) sum_m w_m sum_b b'_b L_{m + e_c + e_b}
    //   dPsi_c   = (1/s)   sum_m La_{m + e_c} w_m
    const int c = k - 1;
    const float bx = ab.y, by = ab.z, bz = ab.w;
    float gq = 0.0f, gp = 0.0f, hb = 0.0f;
#pragma unroll
    for (int nm = 0; nm + 1 < P; ++nm)
#pragma unroll
        for (int ma = nm; ma >= 0; --ma)
#pragma unroll
            for (int mb = nm - ma; mb >= 0; --mb) {
                const int mc = nm - ma - mb;
                const float wm = w[MI<P>::idx(ma, mb, mc)];
                const int i1 = c == 0 ? MI<P>::idx(ma + 1, mb, mc)
                                      : (c == 1 ? MI<P>::idx(ma, mb + 1, mc) : MI<P>::idx(ma, mb, mc + 1));
                gq = fmaf(Lq[i1], wm, gq);
                gp = fmaf(Lp[i1], wm, gp);
                if (nm + 2 < P) {
                    const int ix = c == 0 ? MI<P>::idx(ma + 2, mb, mc)
                                          : (c == 1 ? MI<P>::idx(ma + 1, mb + 1, mc) : MI<P>::idx(ma + 1, mb, mc + 1));
                    const int iy = c == 0 ? MI<P>::idx(ma + 1, mb + 1, mc)
                                          : (c == 1 ? MI<P>::idx(ma, mb + 2, mc) : MI<P>::idx(ma, mb + 1, mc + 1));
                    const int iz = c == 0 ? MI<P>::idx(ma + 1, mb, mc + 1)
                                          : (c == 1 ? MI<P>::idx(ma, mb + 1, mc + 1) : MI<P>::idx(ma, mb, mc + 2));
                    hb = fmaf(wm, fmaf(bz, Lq[iz], fmaf(by, Lq[iy], bx * Lq[ix])), hb);
                }
            }
    v += fmaf(ab.x * gq + p.w * gp, inv_s, hb * inv_s * inv_s);
    if (dx) dx[3 * (int64_t)perm[sidx] + c] = v * dx_scale;
}

template <int P> static int adjoint_p2p_impl(Handle &h, float *dq, float *dx)
{
    FMM_TRY(ensure_full_runs(h));
    static bool configured[64] = {};
    if (h.device >= 0 && h.device < 64 && !configured[h.device]) {
        FMM_CUDA(cudaFuncSetAttribute(k_p2p_adj<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAdjSmem));
        configured[h.device] = true;
    }
    const double ih = 1.0 / h.norm_host[3];
    const int blocks = ceil_div((int64_t)h.n_adj_items * 32, kAdjThreads);
    ++h.launches;
    k_p2p_adj<P><<<blocks, kAdjThreads, kAdjSmem, h.stream>>>(
        (int)h.n_adj_items, h.adj_items.as<int4>(), h.p2p_poff.as<unsigned>(), h.p2p_ent.as<float4>(),
        h.p2p_cnt.as<int>(), h.pos.as<float4>(), h.adj.as<float4>(), h.c_pbeg.as<int>(), h.c_pcnt.as<int>(),
        h.c_level.as<int>(), h.c_parent.as<int>(), h.c_geom.as<float4>(), h.L.as<float>(), h.La.as<float>(),
        h.perm.as<int>(), (float)ih, (float)(ih * ih), dq, dx);
    FMM_CHECK_LAUNCH("adjoint p2p");
    return FMM_OK;
}

int adjoint_p2p(Handle &h, float *dq, float *dx)
{
    if (!h.adj_items_ready) {
        FMM_TRY(build_work_items(h, kAdjG, h.adj_items, h.n_adj_items));
        h.adj_items_ready = true;
    }
    switch (h.P) {
    case 3: return adjoint_p2p_impl<3>(h, dq, dx);
    case 4: return adjoint_p2p_impl<4>(h, dq, dx);
    case 5: return adjoint_p2p_impl<5>(h, dq, dx);
    case 6: return adjoint_p2p_impl<6>(h, dq, dx);
    case 8: return adjoint_p2p_impl<8>(h, dq, dx);
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED;
    }
}

}  // namespace fmm
