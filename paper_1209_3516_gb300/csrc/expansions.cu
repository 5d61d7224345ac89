// expansions.cu -- Cartesian Taylor expansion kernels: P2M, M2M, M2L, L2L.
//
// Sec. 3.1 (Table 1): Cartesian Taylor expansions, O(p^3) coefficients and an
// O(p^6) M2L; Sec. 3.2 names the operators P2M, M2M, M2L, L2L and L2P (L2P is
// fused into the P2P kernel).  The centre of expansion of every cell is its
// geometric centre (Table 2).  Coefficients are stored cell-size scaled (see
// mi.cuh): every cell's multipole and local expansion is a vector of
// T = P(P+1)(P+2)/6 floats, padded to TP, at M[c * TP] and L[c * TP].
//
// Kernel layout:
//   P2M  one warp per leaf, lanes over its particles, warp reduction;
//   M2M  one thread per cell of a level (P <= 6) or one warp per cell over a
//        term table (P = 8), summing its children (bottom-up);
//   M2L  one warp per target cell, lanes over its M2L sources, each lane
//        computing the kernel derivatives D_m(R) of its pair and contracting,
//        then a warp reduction of the T local coefficients;
//   L2L  one thread per cell of a level, from its parent (top-down).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "device_util.cuh"
#include "fmm_internal.cuh"
#include "mi.cuh"

namespace fmm {

// Reduce a T-vector across the warp; every lane ends with the sums.
template <int T> __device__ __forceinline__ void warp_reduce_vec(float *v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < T; ++i) v[i] += __shfl_xor_sync(kFull, v[i], o);
}

// Write a T-vector (held by every lane) to dst[0..TP), lanes striding.
template <int T, int TP> __device__ __forceinline__ void warp_store_vec(const float *v, float *dst)
{
    const int lane = (int)lane_id();
#pragma unroll
    for (int i = 0; i < TP; ++i)
        if ((i & 31) == lane) dst[i] = i < T ? v[i] : 0.0f;
}

// ---------------------------------------------------------------------------
// P2M: Mb_k(C) = sum_j q_j w_k((X_C - u_j) / s_C)
// ---------------------------------------------------------------------------
template <int P>
__global__ void k_p2m(int nleaves, const int *leaf_list, const int *pbeg, const int *pcnt, const int *level,
                      const int *parent, const float4 *geom, const float4 *pos, float *M)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= nleaves) return;
    const int c = leaf_list[warp];
    const float inv_s = ldexpf(1.0f, level[c]);
    // particles are offsets d from the frame centre X_F (the leaf's parent):
    // (X_C - u) / s = (X_C - X_F) / s - d / s, the first term exactly 0 or +-1
    const int fr = parent[c] >= 0 ? parent[c] : c;
    const float4 Xc = geom[c], Xf = geom[fr];
    const float ox = (Xc.x - Xf.x) * inv_s, oy = (Xc.y - Xf.y) * inv_s, oz = (Xc.z - Xf.z) * inv_s;
    float acc[T];
#pragma unroll
    for (int i = 0; i < T; ++i) acc[i] = 0.0f;
    const int b = pbeg[c], e = b + pcnt[c];
    for (int j = b + (int)lane_id(); j < e; j += 32) {
        const float4 p = pos[j];
        float w[T];
        taylor_monomials<P>(fmaf(-p.x, inv_s, ox), fmaf(-p.y, inv_s, oy), fmaf(-p.z, inv_s, oz), w);
#pragma unroll
        for (int i = 0; i < T; ++i) acc[i] = fmaf(p.w, w[i], acc[i]);
    }
    warp_reduce_vec<T>(acc);
    warp_store_vec<T, TP>(acc, M + (size_t)c * TP);
}

// ---------------------------------------------------------------------------
// M2M: Mb_k(P) = sum_{m <= k} Mb_m(C) 2^-|m| w_{k-m}((X_P - X_C) / s_P)
// (child half-width s_C = s_P / 2, (X_P - X_C) / s_P = -(+-1/2) per axis)
// ---------------------------------------------------------------------------
// P <= 6: one thread per cell of a level, fully unrolled.
template <int P>
__global__ void k_m2m(int lo, int n, const int *cbeg, const int *ccnt, const float4 *geom, float *M)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = lo + i;
    const int nch = ccnt[c];
    if (nch == 0) return;   // leaf: its multipole comes from P2M
    const float4 Xp = geom[c];
    float acc[T];
#pragma unroll
    for (int t = 0; t < T; ++t) acc[t] = 0.0f;
    for (int k = 0; k < nch; ++k) {
        const int ch = cbeg[c] + k;
        const float4 Xc = geom[ch];
        float w[T];
        taylor_monomials<P>(Xc.x > Xp.x ? -0.5f : 0.5f, Xc.y > Xp.y ? -0.5f : 0.5f, Xc.z > Xp.z ? -0.5f : 0.5f, w);
        float mc[T];
        const float *src = M + (size_t)ch * TP;
#pragma unroll
        for (int t = 0; t < T; ++t) mc[t] = src[t];
#pragma unroll
        for (int nk = 0; nk < P; ++nk)
#pragma unroll
            for (int ka = nk; ka >= 0; --ka)
#pragma unroll
                for (int kb = nk - ka; kb >= 0; --kb) {
                    const int kc = nk - ka - kb;
                    float s = 0.0f;
#pragma unroll
                    for (int ma = 0; ma <= ka; ++ma)
#pragma unroll
                        for (int mb = 0; mb <= kb; ++mb)
#pragma unroll
                            for (int mc_ = 0; mc_ <= kc; ++mc_) {
                                const float scale = 1.0f / (float)(1 << (ma + mb + mc_));
                                s = fmaf(mc[MI<P>::idx(ma, mb, mc_)] * scale, w[MI<P>::idx(ka - ma, kb - mb, kc - mc_)], s);
                            }
                    acc[MI<P>::idx(ka, kb, kc)] += s;
                }
    }
    float *dst = M + (size_t)c * TP;
#pragma unroll
    for (int t = 0; t < TP; ++t) dst[t] = t < T ? acc[t] : 0.0f;
}

// Higher orders: one warp per cell, lanes over the terms (k, m) of the shift
// from a term table.  With s the child's octant signs, the factor of a term is
// 2^-|k| prod_i (-s_i)^(j_i) / j_i!, j = k - m: the table holds k, m, the parity
// of j per axis and 1/j!; the sign and 2^-|k| are applied here.  The table is
// ordered m-major, so the 32 lanes of a step add into distinct outputs k of a
// shared-memory accumulator.
struct M2MTerm {
    unsigned kmp;   // k | m << 8 | (j_x odd, j_y odd, j_z odd) << 16
    float coef;     // 1 / (j_x! j_y! j_z!)
};

template <int P>
__global__ void __launch_bounds__(128) k_m2m_table(int lo, int n, const int *cbeg, const int *ccnt,
                                                   const float4 *geom, const M2MTerm *terms, int nterms, float *M)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    __shared__ float acc_s[4][TP];
    const int w = threadIdx.x >> 5;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = (int)lane_id();
    if (i >= n) return;
    const int c = lo + i;
    const int nch = ccnt[c];
    if (nch == 0) return;
    float *acc = acc_s[w];
    for (int k = lane; k < TP; k += 32) acc[k] = 0.0f;
    __syncwarp();
    const float4 Xp = geom[c];
    for (int q = 0; q < nch; ++q) {
        const int ch = cbeg[c] + q;
        const float4 Xc = geom[ch];
        const unsigned flip = (Xc.x > Xp.x ? 1u : 0u) | (Xc.y > Xp.y ? 2u : 0u) | (Xc.z > Xp.z ? 4u : 0u);
        const float *mc = M + (size_t)ch * TP;
        for (int t = lane; t < nterms; t += 32) {
            const M2MTerm e = terms[t];
            const unsigned k = e.kmp & 0xffu, m = (e.kmp >> 8) & 0xffu, par = e.kmp >> 16;
            const float v = __ldg(mc + m) * ((__popc(par & flip) & 1) ? -e.coef : e.coef);
            atomicAdd(acc + k, v);
        }
    }
    __syncwarp();
    float *dst = M + (size_t)c * TP;
    for (int k = lane; k < TP; k += 32) {
        if (k < T) {
            int n_deg = 0;
            while ((n_deg + 1) * (n_deg + 2) * (n_deg + 3) / 6 <= k) ++n_deg;
            dst[k] = ldexpf(acc[k], -n_deg);
        } else {
            dst[k] = 0.0f;
        }
    }
}

// Host: the term table of order P, m-major.
static std::vector<M2MTerm> m2m_term_table(int P)
{
    auto idx = [](int a, int b, int c) {
        const int n = a + b + c, bc = b + c;
        return n * (n + 1) * (n + 2) / 6 + bc * (bc + 1) / 2 + c;
    };
    double fact[16];
    fact[0] = 1.0;
    for (int i = 1; i < 16; ++i) fact[i] = fact[i - 1] * i;
    std::vector<M2MTerm> out;
    for (int mn = 0; mn < P; ++mn)
        for (int ma = mn; ma >= 0; --ma)
            for (int mb = mn - ma; mb >= 0; --mb) {
                const int mc = mn - ma - mb;
                for (int kn = mn; kn < P; ++kn)
                    for (int ka = kn; ka >= 0; --ka)
                        for (int kb = kn - ka; kb >= 0; --kb) {
                            const int kc = kn - ka - kb;
                            if (ka < ma || kb < mb || kc < mc) continue;
                            const int ja = ka - ma, jb = kb - mb, jc = kc - mc;
                            M2MTerm e;
                            e.kmp = (unsigned)idx(ka, kb, kc) | ((unsigned)idx(ma, mb, mc) << 8) |
                                    ((unsigned)((ja & 1) | ((jb & 1) << 1) | ((jc & 1) << 2)) << 16);
                            e.coef = (float)(1.0 / (fact[ja] * fact[jb] * fact[jc]));
                            out.push_back(e);
                        }
            }
    return out;
}

// ---------------------------------------------------------------------------
// M2L: Lb_n(T) = (1/s_T) sum_S sum_k (s_S/s_T)^|k| Mb_k(S) D_{n+k}((X_T - X_S)/s_T)
// One warp per target cell, lanes over its M2L sources; each lane computes the
// kernel derivatives of its pair and contracts them with the source multipole
// into the output coefficients N0 <= idx(n) < N1 (all of them for P <= 6; for
// P = 8 two passes over the sources, each recomputing D, keep everything in
// registers), then the warp sums its lanes.
// ---------------------------------------------------------------------------
template <int P, int N0, int N1>
__device__ __forceinline__ void m2l_pass(int t, const int *off, const int *src, const int *level, const float4 *geom,
                                         const float *M, float *L)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP, NO = N1 - N0;
    const float4 Xt = geom[t];
    const int lt = level[t];
    const float inv_st = ldexpf(1.0f, lt);
    float acc[NO];
#pragma unroll
    for (int i = 0; i < NO; ++i) acc[i] = 0.0f;
    const int b = off[t], e = off[t + 1];
    for (int k = b + (int)lane_id(); k < e; k += 32) {
        const int s = src[k];
        const float4 Xs = geom[s];
        float D[T];
        laplace_derivatives<P>((Xt.x - Xs.x) * inv_st, (Xt.y - Xs.y) * inv_st, (Xt.z - Xs.z) * inv_st, D);
        const float rho = ldexpf(1.0f, lt - level[s]);   // s_S / s_T
        float rho_pow[P];
        rho_pow[0] = 1.0f;
#pragma unroll
        for (int d = 1; d < P; ++d) rho_pow[d] = rho_pow[d - 1] * rho;
        m2l_contract_range<P, N0, N1>(reinterpret_cast<const float4 *>(M + (size_t)s * TP), rho_pow, D, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < NO; ++i) acc[i] += __shfl_xor_sync(kFull, acc[i], o);
    float *dst = L + (size_t)t * TP;
    const int lane = (int)lane_id();
#pragma unroll
    for (int i = 0; i < NO; ++i)
        if ((i & 31) == lane) dst[N0 + i] = acc[i] * inv_st;
    if (N1 == T)
        for (int i = T + lane; i < TP; i += 32) dst[i] = 0.0f;
}

template <int P>
__global__ void __launch_bounds__(128) k_m2l(int ncells, const int *off, const int *src, const int *level,
                                             const float4 *geom, const float *M, float *L)
{
    constexpr int T = MI<P>::T;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= ncells) return;
    if constexpr (P >= 8) {
        constexpr int split = MI<P>::idx(5, 0, 0);   // outputs of degree <= 4 | degree >= 5
        m2l_pass<P, 0, split>(t, off, src, level, geom, M, L);
        m2l_pass<P, split, T>(t, off, src, level, geom, M, L);
    } else {
        m2l_pass<P, 0, T>(t, off, src, level, geom, M, L);
    }
}

// ---------------------------------------------------------------------------
// L2L: Lb_k(C) += 2^-|k| sum_{|k+m| <= P-1} Lb_{k+m}(P) w_m((X_C - X_P) / s_P)
// ---------------------------------------------------------------------------
template <int P>
__global__ void k_l2l(int lo, int n, const int *parent, const float4 *geom, float *L)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = lo + i;
    const int p = parent[c];
    const float4 Xc = geom[c], Xp = geom[p];
    float w[T];
    taylor_monomials<P>(Xc.x > Xp.x ? 0.5f : -0.5f, Xc.y > Xp.y ? 0.5f : -0.5f, Xc.z > Xp.z ? 0.5f : -0.5f, w);
    float lp[T];
    const float *sp = L + (size_t)p * TP;
#pragma unroll
    for (int t = 0; t < T; ++t) lp[t] = sp[t];
    float *dst = L + (size_t)c * TP;
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
                dst[id] += s * (1.0f / (float)(1 << nk));
            }
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------
__global__ void k_gather_q(int64_t n, const int *perm, const float *q, float4 *pos)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) pos[s].w = q[perm[s]];
}

template <int P> static int upward_impl(Handle &h, const float *q)
{
    const int nl = (int)h.nleaves;
    ++h.launches;
    k_gather_q<<<ceil_div(h.N, 256), 256, 0, h.stream>>>(h.N, h.perm.as<int>(), q, h.pos.as<float4>());
    ++h.launches;
    k_p2m<P><<<ceil_div((int64_t)nl * 32, 128), 128, 0, h.stream>>>(nl, h.leaf_list.as<int>(), h.c_pbeg.as<int>(),
                                                                    h.c_pcnt.as<int>(), h.c_level.as<int>(),
                                                                    h.c_parent.as<int>(), h.c_geom.as<float4>(),
                                                                    h.pos.as<float4>(), h.M.as<float>());
    if (P >= 8 && h.m2m_nterms == 0) {
        const std::vector<M2MTerm> tab = m2m_term_table(P);
        FMM_TRY(h.m2m_terms.reserve(tab.size() * sizeof(M2MTerm)));
        FMM_CUDA(cudaMemcpy(h.m2m_terms.p, tab.data(), tab.size() * sizeof(M2MTerm), cudaMemcpyHostToDevice));
        h.m2m_nterms = (int)tab.size();
    }
    const int nterms = h.m2m_nterms;
    for (int l = h.nlevels - 2; l >= 0; --l) {
        const int lo = (int)h.level_off[l], n = (int)(h.level_off[l + 1] - h.level_off[l]);
        ++h.launches;
        if (P >= 8)
            k_m2m_table<P><<<ceil_div((int64_t)n * 32, 128), 128, 0, h.stream>>>(
                lo, n, h.c_cbeg.as<int>(), h.c_ccnt.as<int>(), h.c_geom.as<float4>(), h.m2m_terms.as<M2MTerm>(),
                nterms, h.M.as<float>());
        else
            k_m2m<P><<<ceil_div(n, 64), 64, 0, h.stream>>>(lo, n, h.c_cbeg.as<int>(), h.c_ccnt.as<int>(),
                                                           h.c_geom.as<float4>(), h.M.as<float>());
    }
    FMM_CHECK_LAUNCH("upward pass");
    return FMM_OK;
}

template <int P> static int m2l_impl(Handle &h)
{
    const int nc = (int)h.ncells;
    ++h.launches;
    k_m2l<P><<<ceil_div((int64_t)nc * 32, 128), 128, 0, h.stream>>>(nc, h.m2l_off.as<int>(), h.m2l_src.as<int>(),
                                                                    h.c_level.as<int>(), h.c_geom.as<float4>(),
                                                                    h.M.as<float>(), h.L.as<float>());
    FMM_CHECK_LAUNCH("m2l");
    return FMM_OK;
}

template <int P> static int downward_impl(Handle &h)
{
    for (int l = 1; l < h.nlevels; ++l) {
        const int lo = (int)h.level_off[l], n = (int)(h.level_off[l + 1] - h.level_off[l]);
        ++h.launches;
        k_l2l<P><<<ceil_div(n, 64), 64, 0, h.stream>>>(lo, n, h.c_parent.as<int>(), h.c_geom.as<float4>(),
                                                       h.L.as<float>());
    }
    FMM_CHECK_LAUNCH("downward pass");
    return FMM_OK;
}

#define FMM_DISPATCH_P(P, CALL)                                               \
    switch (P) {                                                              \
    case 3: return CALL<3>;                                                   \
    case 4: return CALL<4>;                                                   \
    case 5: return CALL<5>;                                                   \
    case 6: return CALL<6>;                                                   \
    case 8: return CALL<8>;                                                   \
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED; \
    }

int evaluate_upward(Handle &h, const float *q)
{
    FMM_TRY(h.M.reserve((size_t)h.ncells * h.TP * sizeof(float)));
    switch (h.P) {
    case 3: return upward_impl<3>(h, q);
    case 4: return upward_impl<4>(h, q);
    case 5: return upward_impl<5>(h, q);
    case 6: return upward_impl<6>(h, q);
    case 8: return upward_impl<8>(h, q);
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED;
    }
}

int evaluate_m2l(Handle &h)
{
    FMM_TRY(h.L.reserve((size_t)h.ncells * h.TP * sizeof(float)));
    switch (h.P) {
    case 3: return m2l_impl<3>(h);
    case 4: return m2l_impl<4>(h);
    case 5: return m2l_impl<5>(h);
    case 6: return m2l_impl<6>(h);
    case 8: return m2l_impl<8>(h);
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED;
    }
}

int evaluate_downward(Handle &h)
{
    switch (h.P) {
    case 3: return downward_impl<3>(h);
    case 4: return downward_impl<4>(h);
    case 5: return downward_impl<5>(h);
    case 6: return downward_impl<6>(h);
    case 8: return downward_impl<8>(h);
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED;
    }
}

}  // namespace fmm
