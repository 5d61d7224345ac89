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
//   M2M  one warp per cell of a level: three one-dimensional shifts of all its
//        children at once, then their sum (bottom-up);
//   M2L  one warp per target cell, lanes over its M2L sources, each lane
//        computing the kernel derivatives D_m(R) of its pair and contracting,
//        then a warp reduction of the T local coefficients (at P = 8 in two
//        launches, each owning half of the output coefficients);
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

template <int N> struct Pad32Pow2 {   // smallest 32 * 2^j >= N
    static constexpr int value = N <= 32 ? 32 : N <= 64 ? 64 : N <= 128 ? 128 : 256;
};
template <int N> struct ScatterLen {  // array length warp_reduce_scatter<N> needs
    static constexpr int value = N > Pad32Pow2<N>::value / 2 ? N : Pad32Pow2<N>::value / 2;
};

// Sum N values across the warp by recursive halving over V = Pad32Pow2<N>
// slots (slots >= N are zero): on return lane l holds the sums of slots
// [K l, K l + K) in v[0..K), K = V / 32.  Costs about V shuffles instead of
// 5 N for a butterfly on every value.  v must hold ScatterLen<N> floats.
template <int N> __device__ __forceinline__ void warp_reduce_scatter(float *v)
{
    constexpr int V = Pad32Pow2<N>::value;
    const unsigned lane = lane_id();
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        const int half = V >> (step + 1);
        const unsigned mask = 16u >> step;
        const bool upper = (lane & mask) != 0u;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float lo = (step > 0 || i < N) ? v[i] : 0.0f;
            const float hi = (step > 0 || i + half < N) ? v[i + half] : 0.0f;
            const float send = upper ? lo : hi;
            const float keep = upper ? hi : lo;
            v[i] = keep + __shfl_xor_sync(kFull, send, mask);
        }
    }
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
// With kDipole (adjoint sources, adj[j] = (a_j, p_j)): charges a_j and dipoles
// p_j, whose multipole is p . grad_u of a unit charge's:
//   Mb_k(C) += a_j w_k(v_j) - (1/s_C) sum_c p_{j,c} w_{k - e_c}(v_j),  v_j = (X_C - u_j) / s_C.
// ---------------------------------------------------------------------------
template <int P, bool kDipole>
__global__ void k_p2m(int nleaves, const int *leaf_list, const int *pbeg, const int *pcnt, const int *level,
                      const int *parent, const float4 *geom, const float4 *pos, const float4 *adj, float *M)
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
    float acc[ScatterLen<T>::value];
#pragma unroll
    for (int i = 0; i < ScatterLen<T>::value; ++i) acc[i] = 0.0f;
    const int b = pbeg[c], e = b + pcnt[c];
    for (int j = b + (int)lane_id(); j < e; j += 32) {
        const float4 p = pos[j];
        float w[T];
        taylor_monomials<P>(fmaf(-p.x, inv_s, ox), fmaf(-p.y, inv_s, oy), fmaf(-p.z, inv_s, oz), w);
        if constexpr (kDipole) {
            const float4 ab = adj[j];
            const float px = -ab.y * inv_s, py = -ab.z * inv_s, pz = -ab.w * inv_s;
#pragma unroll
            for (int n = 0; n < P; ++n)
#pragma unroll
                for (int ka = n; ka >= 0; --ka)
#pragma unroll
                    for (int kb = n - ka; kb >= 0; --kb) {
                        const int kc = n - ka - kb;
                        const int i = MI<P>::idx(ka, kb, kc);
                        float v = ab.x * w[i];
                        if (ka > 0) v = fmaf(px, w[MI<P>::idx(ka - 1, kb, kc)], v);
                        if (kb > 0) v = fmaf(py, w[MI<P>::idx(ka, kb - 1, kc)], v);
                        if (kc > 0) v = fmaf(pz, w[MI<P>::idx(ka, kb, kc - 1)], v);
                        acc[i] += v;
                    }
        } else {
#pragma unroll
            for (int i = 0; i < T; ++i) acc[i] = fmaf(p.w, w[i], acc[i]);
        }
    }
    if constexpr (T <= 64) {
        constexpr int K = Pad32Pow2<T>::value / 32;
        warp_reduce_scatter<T>(acc);
        float *dst = M + (size_t)c * TP;
        const int lane = (int)lane_id();
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (K * lane + j < TP) dst[K * lane + j] = K * lane + j < T ? acc[j] : 0.0f;
    } else {
        warp_reduce_vec<T>(acc);
        warp_store_vec<T, TP>(acc, M + (size_t)c * TP);
    }
}

// ---------------------------------------------------------------------------
// M2M: Mb_k(P) = sum_{m <= k} Mb_m(C) 2^-|m| w_{k-m}((X_P - X_C) / s_P)
// (child half-width s_C = s_P / 2, (X_P - X_C) / s_P = -(+-1/2) per axis)
// ---------------------------------------------------------------------------
// Storage index of (a, b, c) and its inverse (degree-graded order of mi.cuh).
__device__ __forceinline__ int mi_index(int a, int b, int c)
{
    const int n = a + b + c, bc = b + c;
    return n * (n + 1) * (n + 2) / 6 + bc * (bc + 1) / 2 + c;
}

__device__ __forceinline__ void mi_decode(int i, int &a, int &b, int &c)
{
    int n = 0;
    while ((n + 1) * (n + 2) * (n + 3) / 6 <= i) ++n;
    const int r = i - n * (n + 1) * (n + 2) / 6;   // position inside degree n
    int bc = 0;                                    // b + c = n - a
    while ((bc + 1) * (bc + 2) / 2 <= r) ++bc;
    c = r - bc * (bc + 1) / 2;
    b = bc - c;
    a = n - bc;
}

// Higher orders: the shift is separable.  With s the child's octant signs,
//   Mb_k(P) = 2^-|k| sum_{m <= k} Mb_m(C) prod_i (-s_i)^(k_i - m_i) / (k_i - m_i)!,
// i.e. three one-dimensional shifts (along x, then y, then z), each
//   A_k = sum_{j = 0..k_i} B_{k - j e_i} (-s_i)^j / j!,
// which read only lower indices of the same truncated set.  One block per
// parent cell; all of its children are shifted at once: the work items of a
// pass are the (child, coefficient) pairs, spread over the block's threads,
// with the children's coefficients, the decoded multi-indices and the per-axis
// factors in shared memory (no division, no dependence between children).  A
// block rather than a warp per parent: the upper levels hold a handful of
// parents, and one warp walking its ~3 x 30 work items per pass serially took
// ~40 us per level whatever the level's size.
constexpr int kM2MThreads = 128;

template <int P>
__global__ void __launch_bounds__(kM2MThreads) k_m2m_sep(int lo, const int *cbeg, const int *ccnt,
                                                         const float4 *geom, float *M)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP;
    __shared__ float buf_s[2][8][T];
    __shared__ float fac_s[8][3][P];   // (-s_i)^j / j! per child and axis
    __shared__ unsigned char abc_s[T][4];   // multi-index (a, b, c, |k|) of each storage index
    const int c = lo + (int)blockIdx.x;
    const int nch = ccnt[c];
    if (nch == 0) return;   // leaf (the whole block): its multipole comes from P2M
    const int tid = (int)threadIdx.x;
    for (int k = tid; k < T; k += kM2MThreads) {
        int a, b, cc;
        mi_decode(k, a, b, cc);
        abc_s[k][0] = (unsigned char)a;
        abc_s[k][1] = (unsigned char)b;
        abc_s[k][2] = (unsigned char)cc;
        abc_s[k][3] = (unsigned char)(a + b + cc);
    }
    const int cb = cbeg[c];
    const float4 Xp = geom[c];
    float(*A)[T] = buf_s[0];
    float(*B)[T] = buf_s[1];
    for (int e = tid; e < nch * 3 * P; e += kM2MThreads) {
        const int ch = e / (3 * P), ax = (e / P) % 3, j = e % P;
        const float4 Xc = geom[cb + ch];
        const float pc = ax == 0 ? Xc.x : (ax == 1 ? Xc.y : Xc.z), pp = ax == 0 ? Xp.x : (ax == 1 ? Xp.y : Xp.z);
        float f = 1.0f;
        const float sgn = pc > pp ? -1.0f : 1.0f;
        for (int d = 1; d <= j; ++d) f *= sgn * (1.0f / (float)d);   // constant per call: d <= 7
        fac_s[ch][ax][j] = f;
    }
    for (int e = tid; e < nch * T; e += kM2MThreads) {
        const int ch = e / T, k = e % T;
        A[ch][k] = M[(size_t)(cb + ch) * TP + k];
    }
    __syncthreads();
    // three passes: x (A -> B), y (B -> A), z (A -> B)
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        float(*src)[T] = (ax == 1) ? B : A;
        float(*dst)[T] = (ax == 1) ? A : B;
        for (int e = tid; e < nch * T; e += kM2MThreads) {
            const int ch = e / T, k = e % T;
            const int ka = abc_s[k][0], kb = abc_s[k][1], kc = abc_s[k][2];
            const int kx = ax == 0 ? ka : (ax == 1 ? kb : kc);
            const float *f = fac_s[ch][ax];
            float t = 0.0f;
#pragma unroll
            for (int d = 0; d < P; ++d) {
                if (d > kx) break;
                const int ia = ax == 0 ? ka - d : ka, ib = ax == 1 ? kb - d : kb, ic = ax == 2 ? kc - d : kc;
                t = fmaf(src[ch][mi_index(ia, ib, ic)], f[d], t);
            }
            dst[ch][k] = t;
        }
        __syncthreads();
    }
    // sum over the children, scale by 2^-|k|
    float *out = M + (size_t)c * TP;
    for (int k = tid; k < TP; k += kM2MThreads) {
        float s = 0.0f;
        if (k < T) {
            for (int ch = 0; ch < nch; ++ch) s += B[ch][k];
            s *= 1.0f / (float)(1 << abc_s[k][3]);
        }
        out[k] = s;
    }
}

// ---------------------------------------------------------------------------
// M2L: Lb_n(T) = (1/s_T) sum_S sum_k (s_S/s_T)^|k| Mb_k(S) D_{n+k}((X_T - X_S)/s_T),
// evaluated in its harmonic reduction (mi.cuh, HI): every multipole is folded
// once onto its k_z <= 1 components (k_m2l_fold); then one warp per target
// cell, lanes over its M2L sources: each lane computes the derivatives D_m,
// m_z <= 2, of its pair and contracts them with the folded multipole into the
// outputs n_z <= 1; the warp sums its lanes, restores the outputs n_z >= 2
// from the trace identity and writes all T coefficients.  Each lane streams
// its sources' folded rows into a two-stage shared-memory ring with cp.async,
// one chunk of 32 pairs ahead of the contraction.  The two-slice form of the
// full contraction this replaces took 0.65 ms at N = 1M, P = 8, theta = 0.5.
// ---------------------------------------------------------------------------
template <int P> struct HarmLayout {
    static constexpr int F = HI<P>::F;
    static constexpr int Q = (F + 3) / 4;      // float4 of folded coefficients per row
    static constexpr int G4 = Q + 1;           // + (centre, level): one row of Mf, in float4
    static constexpr int FP = 4 * G4;          // row stride of Mf in floats
    static constexpr int R4 = G4 | 1;          // row stride in the ring (odd: lanes' rows in distinct banks)
    static constexpr int kWarps = 4;           // warps (target cells) per block of k_m2l
    static constexpr size_t ring_bytes = (size_t)kWarps * 2 * 32 * R4 * sizeof(float4);
};

// Mf[c] = the multipole of cell c folded onto its components k_z <= 1 by the
// trace identity (from the highest k_z down, each M_k with k_z >= 2 is
// subtracted from M_{k-2e_z+2e_x} and M_{k-2e_z+2e_y}), at fidx(k), then the
// cell's centre and level (as a float) in the row's last float4.
template <int P>
__global__ void k_m2l_fold(int ncells, const float *M, const float4 *geom, const int *level, float *Mf)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP, F = HI<P>::F, FP = HarmLayout<P>::FP;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    float m[T];
    const float *src = M + (size_t)c * TP;
#pragma unroll
    for (int i = 0; i < T; ++i) m[i] = src[i];
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
    float *dst = Mf + (size_t)c * FP;
#pragma unroll
    for (int e = 0; e < P; ++e)
#pragma unroll
        for (int cc = 0; cc <= 1; ++cc)
#pragma unroll
            for (int a = e - cc; a >= 0; --a) {
                if (cc > e) continue;
                const int b = e - cc - a;
                dst[HI<P>::fidx(a, b, cc)] = m[MI<P>::idx(a, b, cc)];
            }
#pragma unroll
    for (int i = F; i < 4 * HarmLayout<P>::Q; ++i) dst[i] = 0.0f;
    const float4 X = geom[c];
    reinterpret_cast<float4 *>(dst)[HarmLayout<P>::Q] = make_float4(X.x, X.y, X.z, (float)level[c]);
}

template <int P>
__global__ void __launch_bounds__(128, 3) k_m2l(int ncells, const int *off, const int *src, const int *level,
                                                const float4 *geom, const float4 *Mf, float *L)
{
    constexpr int T = MI<P>::T, TP = MI<P>::TP, F = HI<P>::F, ND = HI<P>::ND;
    constexpr int Q = HarmLayout<P>::Q, G4 = HarmLayout<P>::G4, R4 = HarmLayout<P>::R4;
    extern __shared__ float4 m2l_ring[];   // [warp][stage][lane][R4]
    __shared__ float sums[HarmLayout<P>::kWarps][HarmLayout<P>::FP];   // the reduced outputs n_z <= 1
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= ncells) return;
    const int lane = (int)lane_id();
    const int w = (threadIdx.x >> 5) % HarmLayout<P>::kWarps;
    float4 *row0 = m2l_ring + ((size_t)w * 2 * 32 + lane) * R4;   // stage 1 at + 32 R4
    const float4 Xt = geom[t];
    const int lt = level[t];
    const float inv_st = ldexpf(1.0f, lt);
    float acc[ScatterLen<F>::value];
#pragma unroll
    for (int i = 0; i < ScatterLen<F>::value; ++i) acc[i] = 0.0f;
    const int b = off[t], e = off[t + 1];
    // lane-private pipeline: the rows of entries b + lane + 32 i, one chunk ahead
    int s = b + lane < e ? src[b + lane] : -1;
    if (s >= 0)
#pragma unroll
        for (int q = 0; q < G4; ++q) cp_async16(row0 + q, Mf + (size_t)s * G4 + q);
    cp_async_commit();
    int sn = b + 32 + lane < e ? src[b + 32 + lane] : -1;
    int stage = 0;
    for (int k0 = b; k0 < e; k0 += 32) {
        float4 *nrow = row0 + (stage ^ 1) * 32 * R4;
        if (sn >= 0)
#pragma unroll
            for (int q = 0; q < G4; ++q) cp_async16(nrow + q, Mf + (size_t)sn * G4 + q);
        cp_async_commit();
        const int snn = k0 + 64 + lane < e ? src[k0 + 64 + lane] : -1;
        if (s >= 0) {
            cp_async_wait_1();
            const float4 *row = row0 + stage * 32 * R4;
            const float4 Xs = row[Q];
            float D[ND];
            laplace_derivatives_z2<P>((Xt.x - Xs.x) * inv_st, (Xt.y - Xs.y) * inv_st, (Xt.z - Xs.z) * inv_st, D);
            const float rho = ldexpf(1.0f, lt - (int)Xs.w);   // s_S / s_T
            float rho_pow[P];
            rho_pow[0] = 1.0f;
#pragma unroll
            for (int d = 1; d < P; ++d) rho_pow[d] = rho_pow[d - 1] * rho;
            m2l_contract_harmonic<P>(row, rho_pow, D, acc);
        }
        s = sn;
        sn = snn;
        stage ^= 1;
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    warp_reduce_scatter<F>(acc);
    float *sw = sums[w];
    constexpr int K = Pad32Pow2<F>::value / 32;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int i = K * lane + j;
        if (i < F) sw[i] = acc[j];
    }
    __syncwarp();
    // every lane: all T outputs, n_z >= 2 from the trace identity, then its share written
    float full[T];
#pragma unroll
    for (int d = 0; d < P; ++d)
#pragma unroll
        for (int cc = 0; cc <= 1; ++cc)
#pragma unroll
            for (int a = d - cc; a >= 0; --a) {
                if (cc > d) continue;
                const int bb = d - cc - a;
                full[MI<P>::idx(a, bb, cc)] = sw[HI<P>::fidx(a, bb, cc)] * inv_st;
            }
#pragma unroll
    for (int z = 2; z < P; ++z)
#pragma unroll
        for (int d = z; d < P; ++d)
#pragma unroll
            for (int a = d - z; a >= 0; --a) {
                const int bb = d - z - a;
                full[MI<P>::idx(a, bb, z)] = -full[MI<P>::idx(a + 2, bb, z - 2)] - full[MI<P>::idx(a, bb + 2, z - 2)];
            }
    warp_store_vec<T, TP>(full, L + (size_t)t * TP);
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

template <int P> static int m2m_levels(Handle &h, float *M)
{
    for (int l = h.nlevels - 2; l >= 0; --l) {
        const int lo = (int)h.level_off[l], n = (int)(h.level_off[l + 1] - h.level_off[l]);
        if (n <= 0) continue;
        ++h.launches;
        k_m2m_sep<P><<<n, kM2MThreads, 0, h.stream>>>(lo, h.c_cbeg.as<int>(), h.c_ccnt.as<int>(),
                                                       h.c_geom.as<float4>(), M);
    }
    FMM_CHECK_LAUNCH("upward pass");
    return FMM_OK;
}

template <int P> static int upward_impl(Handle &h, const float *q)
{
    const int nl = (int)h.nleaves;
    ++h.launches;
    k_gather_q<<<ceil_div(h.N, 256), 256, 0, h.stream>>>(h.N, h.perm.as<int>(), q, h.pos.as<float4>());
    ++h.launches;
    k_p2m<P, false><<<ceil_div((int64_t)nl * 32, 128), 128, 0, h.stream>>>(
        nl, h.leaf_list.as<int>(), h.c_pbeg.as<int>(), h.c_pcnt.as<int>(), h.c_level.as<int>(), h.c_parent.as<int>(),
        h.c_geom.as<float4>(), h.pos.as<float4>(), nullptr, h.M.as<float>());
    return m2m_levels<P>(h, h.M.as<float>());
}

// adj[s] = (dphi[perm[s]], dgrad[perm[s]] / h): charges and dipoles of the adjoint
// field in normalised coordinates (either input may be absent: zero)
__global__ void k_gather_adj(int64_t n, const int *perm, const float *dphi, const float *dgrad, float inv_h,
                             float4 *adj)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int64_t i = perm[s];
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (dphi) v.x = dphi[i];
    if (dgrad) {
        v.y = dgrad[3 * i] * inv_h;
        v.z = dgrad[3 * i + 1] * inv_h;
        v.w = dgrad[3 * i + 2] * inv_h;
    }
    adj[s] = v;
}

template <int P> static int adjoint_upward_impl(Handle &h, const float *dphi, const float *dgrad)
{
    const int nl = (int)h.nleaves;
    ++h.launches;
    k_gather_adj<<<ceil_div(h.N, 256), 256, 0, h.stream>>>(h.N, h.perm.as<int>(), dphi, dgrad,
                                                          (float)(1.0 / h.norm_host[3]), h.adj.as<float4>());
    ++h.launches;
    k_p2m<P, true><<<ceil_div((int64_t)nl * 32, 128), 128, 0, h.stream>>>(
        nl, h.leaf_list.as<int>(), h.c_pbeg.as<int>(), h.c_pcnt.as<int>(), h.c_level.as<int>(), h.c_parent.as<int>(),
        h.c_geom.as<float4>(), h.pos.as<float4>(), h.adj.as<float4>(), h.Ma.as<float>());
    return m2m_levels<P>(h, h.Ma.as<float>());
}

template <int P> static int m2l_impl(Handle &h, const float *M, float *L)
{
    using HL = HarmLayout<P>;
    const int nc = (int)h.ncells;
    static bool configured[64] = {};
    if (h.device >= 0 && h.device < 64 && !configured[h.device]) {
        FMM_CUDA(cudaFuncSetAttribute(k_m2l<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HL::ring_bytes));
        configured[h.device] = true;
    }
    FMM_TRY(h.Mf.reserve((size_t)nc * HL::FP * sizeof(float)));
    ++h.launches;
    k_m2l_fold<P><<<ceil_div(nc, 128), 128, 0, h.stream>>>(nc, M, h.c_geom.as<float4>(), h.c_level.as<int>(),
                                                          h.Mf.as<float>());
    ++h.launches;
    k_m2l<P><<<ceil_div((int64_t)nc * 32, 32 * HL::kWarps), 32 * HL::kWarps, HL::ring_bytes, h.stream>>>(
        nc, h.m2l_off.as<int>(), h.m2l_src.as<int>(), h.c_level.as<int>(), h.c_geom.as<float4>(),
        h.Mf.as<float4>(), L);
    FMM_CHECK_LAUNCH("m2l");
    return FMM_OK;
}

template <int P> static int downward_impl(Handle &h, float *L)
{
    for (int l = 1; l < h.nlevels; ++l) {
        const int lo = (int)h.level_off[l], n = (int)(h.level_off[l + 1] - h.level_off[l]);
        ++h.launches;
        k_l2l<P><<<ceil_div(n, 64), 64, 0, h.stream>>>(lo, n, h.c_parent.as<int>(), h.c_geom.as<float4>(), L);
    }
    FMM_CHECK_LAUNCH("downward pass");
    return FMM_OK;
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

int evaluate_m2l(Handle &h, const float *M, float *L)
{
    switch (h.P) {
    case 3: return m2l_impl<3>(h, M, L);
    case 4: return m2l_impl<4>(h, M, L);
    case 5: return m2l_impl<5>(h, M, L);
    case 6: return m2l_impl<6>(h, M, L);
    case 8: return m2l_impl<8>(h, M, L);
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED;
    }
}

int evaluate_downward(Handle &h, float *L)
{
    switch (h.P) {
    case 3: return downward_impl<3>(h, L);
    case 4: return downward_impl<4>(h, L);
    case 5: return downward_impl<5>(h, L);
    case 6: return downward_impl<6>(h, L);
    case 8: return downward_impl<8>(h, L);
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED;
    }
}

int adjoint_upward(Handle &h, const float *dphi, const float *dgrad)
{
    FMM_TRY(h.adj.reserve((size_t)h.N * sizeof(float4)));
    FMM_TRY(h.Ma.reserve((size_t)h.ncells * h.TP * sizeof(float)));
    switch (h.P) {
    case 3: return adjoint_upward_impl<3>(h, dphi, dgrad);
    case 4: return adjoint_upward_impl<4>(h, dphi, dgrad);
    case 5: return adjoint_upward_impl<5>(h, dphi, dgrad);
    case 6: return adjoint_upward_impl<6>(h, dphi, dgrad);
    case 8: return adjoint_upward_impl<8>(h, dphi, dgrad);
    default: set_error("expansion order not compiled"); return FMM_ERR_UNSUPPORTED;
    }
}

}  // namespace fmm
