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
//   M2M  one thread per cell of a level, sum over its children (bottom-up);
//   M2L  one warp per target cell, lanes over its M2L sources, each lane
//        computing the kernel derivatives D_m(R) of its pair and contracting,
//        then a warp reduction of the T local coefficients;
//   L2L  one thread per cell of a level, from its parent (top-down).
#include <cuda_runtime.h>

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
        // acc_k += sum_{m <= k} mc_m 2^-|m| w_{k-m}
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

// ---------------------------------------------------------------------------
// M2L: Lb_n(T) = (1/s_T) sum_S sum_k (s_S/s_T)^|k| Mb_k(S) D_{n+k}((X_T - X_S)/s_T)
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(128) k_m2l(int ncells, const int *off, const int *src, const int *level,
                                             const float4 *geom, const float *M, float *L)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= ncells) return;
    const float4 Xt = geom[t];
    const int lt = level[t];
    const float inv_st = ldexpf(1.0f, lt);
    float acc[T];
#pragma unroll
    for (int i = 0; i < T; ++i) acc[i] = 0.0f;
    const int b = off[t], e = off[t + 1];
    for (int k = b + (int)lane_id(); k < e; k += 32) {
        const int s = src[k];
        const float4 Xs = geom[s];
        const float rho = ldexpf(1.0f, lt - level[s]);   // s_S / s_T
        float D[T];
        laplace_derivatives<P>((Xt.x - Xs.x) * inv_st, (Xt.y - Xs.y) * inv_st, (Xt.z - Xs.z) * inv_st, D);
        float Mk[T];
        const float4 *m4 = reinterpret_cast<const float4 *>(M + (size_t)s * TP);
#pragma unroll
        for (int i = 0; i < TP / 4; ++i) {
            const float4 v = __ldg(m4 + i);
            if (4 * i + 0 < T) Mk[4 * i + 0] = v.x;
            if (4 * i + 1 < T) Mk[4 * i + 1] = v.y;
            if (4 * i + 2 < T) Mk[4 * i + 2] = v.z;
            if (4 * i + 3 < T) Mk[4 * i + 3] = v.w;
        }
        if (rho != 1.0f) {
            float r = rho;
#pragma unroll
            for (int nk = 1; nk < P; ++nk) {
#pragma unroll
                for (int i = MI<P>::idx(nk, 0, 0); i < MI<P>::idx(nk, 0, 0) + (nk + 1) * (nk + 2) / 2; ++i)
                    Mk[i] *= r;
                r *= rho;
            }
        }
        m2l_contract<P>(Mk, D, acc);
    }
    warp_reduce_vec<T>(acc);
#pragma unroll
    for (int i = 0; i < T; ++i) acc[i] *= inv_st;
    warp_store_vec<T, TP>(acc, L + (size_t)t * TP);
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
    for (int l = h.nlevels - 2; l >= 0; --l) {
        const int lo = (int)h.level_off[l], n = (int)(h.level_off[l + 1] - h.level_off[l]);
        ++h.launches;
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
