// batch.cu -- many charge vectors on one geometry (fmm_evaluate_batch).
//
// With nrhs <= 32 charge vectors on a fixed tree, every operator of the
// evaluation becomes a contraction over the right-hand sides:
//   P2M, M2M, M2L, L2L  one warp per cell, lane r = right-hand side r: the
//        geometric factors (monomials, kernel derivatives D) are computed once
//        and applied to 32 expansion vectors; expansions are stored
//        Mb[cell][TP][32] so that lanes read consecutive words;
//   P2P + L2P  a dense product on the 5th-generation tensor cores
//        (batch_tc.cu): the charges are gathered here into sorted order and
//        split into BF16 high and low parts.
// The tree, lists and P2P source runs are those of the last build.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "device_util.cuh"
#include "fmm_internal.cuh"
#include "mi.cuh"
#include "p2p_common.cuh"

namespace fmm {

constexpr int kB = 32;              // right-hand sides per batch (lanes)

// ---------------------------------------------------------------------------
// gather: qb[s][r] = q[r][perm[s]] (FP32) and its BF16 split (hi, lo)
// ---------------------------------------------------------------------------
__global__ void k_gather_qbatch(int64_t n, int nrhs, const int *perm, const float *q, float *qb,
                                __nv_bfloat16 *qh, __nv_bfloat16 *ql)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * kB) return;
    const int64_t s = i / kB;
    const int r = (int)(i % kB);
    const float v = r < nrhs ? q[(int64_t)r * n + perm[s]] : 0.0f;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    qb[i] = v;
    qh[i] = hi;
    ql[i] = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// ---------------------------------------------------------------------------
// far field, lanes over right-hand sides
// ---------------------------------------------------------------------------
template <int P>
__global__ void k_p2m_batch(int nleaves, const int *leaf_list, const int *pbeg, const int *pcnt, const int *level,
                            const int *parent, const float4 *geom, const float4 *pos, const float *qb, float *Mb)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= nleaves) return;
    const int r = (int)lane_id();
    const int c = leaf_list[warp];
    const float inv_s = ldexpf(1.0f, level[c]);
    const int fr = parent[c] >= 0 ? parent[c] : c;
    const float4 Xc = geom[c], Xf = geom[fr];
    const float ox = (Xc.x - Xf.x) * inv_s, oy = (Xc.y - Xf.y) * inv_s, oz = (Xc.z - Xf.z) * inv_s;
    float acc[T];
#pragma unroll
    for (int i = 0; i < T; ++i) acc[i] = 0.0f;
    const int b = pbeg[c], e = b + pcnt[c];
    for (int j = b; j < e; ++j) {
        const float4 p = pos[j];
        float w[T];
        taylor_monomials<P>(fmaf(-p.x, inv_s, ox), fmaf(-p.y, inv_s, oy), fmaf(-p.z, inv_s, oz), w);
        const float q = qb[(size_t)j * kB + r];
#pragma unroll
        for (int i = 0; i < T; ++i) acc[i] = fmaf(q, w[i], acc[i]);
    }
    float *dst = Mb + (size_t)c * TP * kB + r;
#pragma unroll
    for (int i = 0; i < TP; ++i) dst[i * kB] = i < T ? acc[i] : 0.0f;
}

template <int P>
__global__ void k_m2m_batch(int lo, int n, const int *cbeg, const int *ccnt, const float4 *geom, float *Mb)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= n) return;
    const int r = (int)lane_id();
    const int c = lo + warp;
    const int nch = ccnt[c];
    if (nch == 0) return;   // leaf: its multipole comes from P2M
    const float4 Xp = geom[c];
    float acc[T];
#pragma unroll
    for (int t = 0; t < T; ++t) acc[t] = 0.0f;
    for (int k = 0; k < nch; ++k) {
        const int ch = cbeg[c] + k;
        const float4 Xc = geom[ch];
        // child multipole, scaled to the parent's cell size: 2^-|m| Mb_m(C)
        float mc[T];
        const float *src = Mb + (size_t)ch * TP * kB + r;
#pragma unroll
        for (int na = 0; na < P; ++na)
#pragma unroll
            for (int a = na; a >= 0; --a)
#pragma unroll
                for (int b = na - a; b >= 0; --b) {
                    const int i = MI<P>::idx(a, b, na - a - b);
                    mc[i] = src[i * kB] * (1.0f / (float)(1 << na));
                }
        // separable shift by (X_P - X_C) / s_P = -+1/2 per axis, one axis at a time:
        // m'_(a,b,c) = sum_{a' <= a} m_(a',b,c) dx^(a-a') / (a-a')!
        const float d[3] = {Xc.x > Xp.x ? -0.5f : 0.5f, Xc.y > Xp.y ? -0.5f : 0.5f, Xc.z > Xp.z ? -0.5f : 0.5f};
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            float pw[P];   // d^j / j!
            pw[0] = 1.0f;
#pragma unroll
            for (int j = 1; j < P; ++j) pw[j] = pw[j - 1] * d[ax] * (1.0f / j);
            // in place, highest power first along the axis so sources are still unshifted
#pragma unroll
            for (int na = P - 1; na >= 0; --na)
#pragma unroll
                for (int a = na; a >= 0; --a)
#pragma unroll
                    for (int b = na - a; b >= 0; --b) {
                        const int cc = na - a - b;
                        const int e[3] = {a, b, cc};
                        const int i = MI<P>::idx(a, b, cc);
                        float s = mc[i];
#pragma unroll
                        for (int j = 1; j <= e[ax]; ++j) {
                            int f[3] = {a, b, cc};
                            f[ax] -= j;
                            s = fmaf(mc[MI<P>::idx(f[0], f[1], f[2])], pw[j], s);
                        }
                        mc[i] = s;
                    }
        }
#pragma unroll
        for (int t = 0; t < T; ++t) acc[t] += mc[t];
    }
    float *dst = Mb + (size_t)c * TP * kB + r;
#pragma unroll
    for (int t = 0; t < TP; ++t) dst[t * kB] = t < T ? acc[t] : 0.0f;
}

// M2L in the harmonic reduction of the single-vector M2L (mi.cuh, HI): the
// multipoles are first folded in place onto their components with k_z <= 1
// (rows fidx(k) of each cell, lane = vector), then one warp per target cell
// computes, per chunk of 32 sources, the derivatives D_m (m_z <= 2) of one
// pair per lane into shared memory, and lane r contracts every pair of the
// chunk with its folded multipole vector r into the outputs n_z <= 1; the
// outputs n_z >= 2 follow from the trace identity in the epilogue.
constexpr int kM2LBatchThreads = 64;

// Mb[c][fidx(k)][r] <- folded multipole of vector r (in place: rows 0 .. F-1).
template <int P>
__global__ void k_m2l_fold_batch(int ncells, float *Mb)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= ncells) return;
    float *cm = Mb + (size_t)c * TP * kB + lane_id();
    float m[T];
#pragma unroll
    for (int i = 0; i < T; ++i) m[i] = cm[i * kB];
#pragma unroll
    for (int z = P - 1; z >= 2; --z)
#pragma unroll
        for (int n = z; n < P; ++n)
#pragma unroll
            for (int a = n - z; a >= 0; --a) {
                const int b = n - z - a;
                const float v = m[MI<P>::idx(a, b, z)];
                m[MI<P>::idx(a + 2, b, z - 2)] -= v;
                m[MI<P>::idx(a, b + 2, z - 2)] -= v;
            }
#pragma unroll
    for (int e = 0; e < P; ++e)
#pragma unroll
        for (int kc = 0; kc <= 1; ++kc)
#pragma unroll
            for (int a = e - kc; a >= 0; --a) {
                if (kc > e) continue;
                const int b = e - kc - a;
                cm[HI<P>::fidx(a, b, kc) * kB] = m[MI<P>::idx(a, b, kc)];
            }
}

template <int P>
__global__ void __launch_bounds__(kM2LBatchThreads) k_m2l_batch(int ncells, const int *off, const int *src,
                                                                const int *level, const float4 *geom, const float *Mb,
                                                                float *Lb)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP, F = HI<P>::F, ND = HI<P>::ND;
    constexpr int W = kM2LBatchThreads / 32;
    __shared__ float Ds[W][32][ND + 1];
    __shared__ float Rho[W][32];
    __shared__ int Src[W][32];
    const int w = threadIdx.x >> 5;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= ncells) return;
    const int lane = (int)lane_id();
    const float4 Xt = geom[t];
    const int lt = level[t];
    const float inv_st = ldexpf(1.0f, lt);
    float acc[F];
#pragma unroll
    for (int i = 0; i < F; ++i) acc[i] = 0.0f;
    const int b = off[t], e = off[t + 1];
    for (int k0 = b; k0 < e; k0 += 32) {
        const int k = k0 + lane;
        if (k < e) {
            const int s = src[k];
            const float4 Xs = geom[s];
            float D[ND];
            laplace_derivatives_z2<P>((Xt.x - Xs.x) * inv_st, (Xt.y - Xs.y) * inv_st, (Xt.z - Xs.z) * inv_st, D);
#pragma unroll
            for (int i = 0; i < ND; ++i) Ds[w][lane][i] = D[i];
            Rho[w][lane] = ldexpf(1.0f, lt - level[s]);
            Src[w][lane] = s;
        }
        __syncwarp();
        const int np = min(32, e - k0);
        for (int j = 0; j < np; ++j) {
            const float *Mj = Mb + (size_t)Src[w][j] * TP * kB + lane;
            const float *D = Ds[w][j];
            const float rho = Rho[w][j];
            float rp = 1.0f;
#pragma unroll
            for (int ke = 0; ke < P; ++ke) {
#pragma unroll
                for (int kc = 0; kc <= 1; ++kc)
#pragma unroll
                    for (int ka = ke - kc; ka >= 0; --ka) {
                        if (kc > ke) continue;
                        const int kb = ke - kc - ka;
                        const float m = Mj[HI<P>::fidx(ka, kb, kc) * kB] * rp;
#pragma unroll
                        for (int d = 0; d + ke < P; ++d)
#pragma unroll
                            for (int nc = 0; nc <= 1; ++nc)
#pragma unroll
                                for (int na = d - nc; na >= 0; --na) {
                                    if (nc > d) continue;
                                    const int nb = d - nc - na;
                                    const int in = HI<P>::fidx(na, nb, nc);
                                    acc[in] = fmaf(m, D[HI<P>::didx(na + ka, nb + kb, nc + kc)], acc[in]);
                                }
                    }
                rp *= rho;
            }
        }
        __syncwarp();
    }
    float full[T];
#pragma unroll
    for (int d = 0; d < P; ++d)
#pragma unroll
        for (int nc = 0; nc <= 1; ++nc)
#pragma unroll
            for (int na = d - nc; na >= 0; --na) {
                if (nc > d) continue;
                const int nb = d - nc - na;
                full[MI<P>::idx(na, nb, nc)] = acc[HI<P>::fidx(na, nb, nc)] * inv_st;
            }
#pragma unroll
    for (int z = 2; z < P; ++z)
#pragma unroll
        for (int d = z; d < P; ++d)
#pragma unroll
            for (int na = d - z; na >= 0; --na) {
                const int nb = d - z - na;
                full[MI<P>::idx(na, nb, z)] = -full[MI<P>::idx(na + 2, nb, z - 2)] - full[MI<P>::idx(na, nb + 2, z - 2)];
            }
    float *dst = Lb + (size_t)t * TP * kB + lane;
#pragma unroll
    for (int i = 0; i < TP; ++i) dst[i * kB] = i < T ? full[i] : 0.0f;
}

template <int P>
__global__ void k_l2l_batch(int lo, int n, const int *parent, const float4 *geom, float *Lb)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= n) return;
    const int r = (int)lane_id();
    const int c = lo + warp;
    const int p = parent[c];
    const float4 Xc = geom[c], Xp = geom[p];
    float w[T];
    taylor_monomials<P>(Xc.x > Xp.x ? 0.5f : -0.5f, Xc.y > Xp.y ? 0.5f : -0.5f, Xc.z > Xp.z ? 0.5f : -0.5f, w);
    float lp[T];
    const float *sp = Lb + (size_t)p * TP * kB + r;
#pragma unroll
    for (int t = 0; t < T; ++t) lp[t] = sp[t * kB];
    float *dst = Lb + (size_t)c * TP * kB + r;
#pragma unroll
    for (int nk = 0; nk < P; ++nk)
#pragma unroll
        for (int ka = nk; ka >= 0; --ka)
#pragma unroll
            for (int kb = nk - ka; kb >= 0; --kb) {
                const int kc = nk - ka - kb;
                float s = 0.0f;
#pragma unroll
                for (int nm = 0; nm + nk < P; ++nm)
#pragma unroll
                    for (int ma = nm; ma >= 0; --ma)
#pragma unroll
                        for (int mb = nm - ma; mb >= 0; --mb) {
                            const int mc = nm - ma - mb;
                            s = fmaf(lp[MI<P>::idx(ka + ma, kb + mb, kc + mc)], w[MI<P>::idx(ma, mb, mc)], s);
                        }
                const int id = MI<P>::idx(ka, kb, kc);
                dst[id * kB] += s * (1.0f / (float)(1 << nk));
            }
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
template <int P> static int batch_impl(Handle &h, const float *q, int nrhs, float *phi, float *grad)
{
    const int64_t N = h.N;
    const int nl = (int)h.nleaves, nc = (int)h.ncells;
    constexpr int TP = MI<P>::TP;
    FMM_TRY(h.qb.reserve((size_t)N * kB * sizeof(float)));
    FMM_TRY(h.qbh.reserve((size_t)N * kB * sizeof(__nv_bfloat16)));
    FMM_TRY(h.qbl.reserve((size_t)N * kB * sizeof(__nv_bfloat16)));
    FMM_TRY(h.Mb.reserve((size_t)nc * TP * kB * sizeof(float)));
    FMM_TRY(h.Lb.reserve((size_t)nc * TP * kB * sizeof(float)));
    float *Mb = h.Mb.as<float>(), *Lb = h.Lb.as<float>();
    phase_begin(h, FMM_PHASE_UPWARD);
    ++h.launches;
    k_gather_qbatch<<<ceil_div(N * kB, 256), 256, 0, h.stream>>>(N, nrhs, h.perm.as<int>(), q, h.qb.as<float>(),
                                                                h.qbh.as<__nv_bfloat16>(), h.qbl.as<__nv_bfloat16>());
    ++h.launches;
    k_p2m_batch<P><<<ceil_div((int64_t)nl * 32, 128), 128, 0, h.stream>>>(
        nl, h.leaf_list.as<int>(), h.c_pbeg.as<int>(), h.c_pcnt.as<int>(), h.c_level.as<int>(), h.c_parent.as<int>(),
        h.c_geom.as<float4>(), h.pos.as<float4>(), h.qb.as<float>(), Mb);
    for (int l = h.nlevels - 2; l >= 0; --l) {
        const int lo = (int)h.level_off[l], n = (int)(h.level_off[l + 1] - h.level_off[l]);
        ++h.launches;
        k_m2m_batch<P><<<ceil_div((int64_t)n * 32, 128), 128, 0, h.stream>>>(lo, n, h.c_cbeg.as<int>(),
                                                                             h.c_ccnt.as<int>(), h.c_geom.as<float4>(), Mb);
    }
    phase_end(h, FMM_PHASE_UPWARD);
    phase_begin(h, FMM_PHASE_M2L);
    ++h.launches;
    k_m2l_fold_batch<P><<<ceil_div((int64_t)nc * 32, 128), 128, 0, h.stream>>>(nc, Mb);
    ++h.launches;
    k_m2l_batch<P><<<ceil_div((int64_t)nc * 32, kM2LBatchThreads), kM2LBatchThreads, 0, h.stream>>>(
        nc, h.m2l_off.as<int>(), h.m2l_src.as<int>(), h.c_level.as<int>(), h.c_geom.as<float4>(), Mb, Lb);
    phase_end(h, FMM_PHASE_M2L);
    phase_begin(h, FMM_PHASE_DOWNWARD);
    for (int l = 1; l < h.nlevels; ++l) {
        const int lo = (int)h.level_off[l], n = (int)(h.level_off[l + 1] - h.level_off[l]);
        ++h.launches;
        k_l2l_batch<P><<<ceil_div((int64_t)n * 32, 128), 128, 0, h.stream>>>(lo, n, h.c_parent.as<int>(),
                                                                             h.c_geom.as<float4>(), Lb);
    }
    phase_end(h, FMM_PHASE_DOWNWARD);
    FMM_CHECK_LAUNCH("batched far field");
    phase_begin(h, FMM_PHASE_P2P);
    FMM_TRY(p2p_batch_tc(h, nrhs, phi, grad));
    phase_end(h, FMM_PHASE_P2P);
    FMM_CHECK_LAUNCH("batched p2p");
    return FMM_OK;
}

int evaluate_batch(Handle &h, const float *q, int nrhs, float *phi, float *grad)
{
    switch (h.P) {
    case 3: return batch_impl<3>(h, q, nrhs, phi, grad);
    case 4: return batch_impl<4>(h, q, nrhs, phi, grad);
    case 5: return batch_impl<5>(h, q, nrhs, phi, grad);
    case 6: return batch_impl<6>(h, q, nrhs, phi, grad);
    case 8: return batch_impl<8>(h, q, nrhs, phi, grad);
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED;
    }
}

}  // namespace fmm
