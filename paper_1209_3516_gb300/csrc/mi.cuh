// mi.cuh -- Cartesian Taylor multi-index arithmetic, fully unrolled for a fixed order P.
//
// Multi-indices k = (a, b, c) with |k| = a + b + c <= P-1 (Sec. 3.1, Table 1:
// Cartesian Taylor expansions, O(p^3) coefficients).  Storage order: by total
// degree n, then a descending, then b descending:
//     idx(a, b, c) = n (n+1) (n+2) / 6 + (n-a) (n-a+1) / 2 + c.
// All loops below have compile-time bounds and are unrolled, so every index is
// a constant and coefficient arrays live in registers.
//
// Scaled conventions of this library (cell half-width s = 2^-level, exact in FP32):
//   multipole  Mb_k(C) = sum_j q_j w_k((X_C - u_j) / s_C),     w_k(v) = v^k / k!
//   local      Lb_n(C) = s_C^|n| * d^n phi / dx^n (X_C)  (so phi = sum_n Lb_n w_n((x - X_C) / s_C))
//   M2L        Lb_n(T) = (1/s_T) sum_k (s_S/s_T)^|k| Mb_k(S) D_{n+k}((X_T - X_S) / s_T)
//   with D_m(R) = d^m (1/|R|) / dR^m the raw derivatives of the Laplace kernel.
// Cell-size scaling keeps every coefficient O(1) at any depth of the tree.
#pragma once

#include <cuda_runtime.h>

#include "device_util.cuh"

namespace fmm {

template <int P> struct MI {
    static constexpr int T = P * (P + 1) * (P + 2) / 6;   // coefficients with |k| <= P-1
    static constexpr int TP = (T + 3) & ~3;              // padded to a float4 multiple
    __host__ __device__ static constexpr int idx(int a, int b, int c)
    {
        return (a + b + c) * (a + b + c + 1) * (a + b + c + 2) / 6 + (b + c) * (b + c + 1) / 2 + c;
    }
};

// w[idx(k)] = v^k / k! for |k| <= P-1 (Taylor monomials).
template <int P>
__device__ __forceinline__ void taylor_monomials(float vx, float vy, float vz, float *w)
{
    float sx[P], sy[P], sz[P];   // v / j, j = 1..P-1 (index j)
#pragma unroll
    for (int j = 1; j < P; ++j) {
        sx[j] = vx * (1.0f / j);
        sy[j] = vy * (1.0f / j);
        sz[j] = vz * (1.0f / j);
    }
    w[0] = 1.0f;
#pragma unroll
    for (int n = 1; n < P; ++n)
#pragma unroll
        for (int a = n; a >= 0; --a)
#pragma unroll
            for (int b = n - a; b >= 0; --b) {
                const int c = n - a - b;
                const int i = MI<P>::idx(a, b, c);
                if (a > 0) w[i] = w[MI<P>::idx(a - 1, b, c)] * sx[a];
                else if (b > 0) w[i] = w[MI<P>::idx(a, b - 1, c)] * sy[b];
                else w[i] = w[MI<P>::idx(a, b, c - 1)] * sz[c];
            }
}

// D[idx(m)] = d^m (1/|R|) / dR^m for |m| <= P-1 (raw Cartesian derivatives).
// Recurrence (multiply the Taylor-coefficient recurrence of Lindsay & Krasny,
// J. Comput. Phys. 172 (2001), by m!):
//   |m| r^2 D_m = -(2|m|-1) sum_i m_i R_i D_{m-e_i} - (|m|-1) sum_i m_i (m_i-1) D_{m-2e_i}.
template <int P>
__device__ __forceinline__ void laplace_derivatives(float Rx, float Ry, float Rz, float *D)
{
    const float r2 = fmaf(Rz, Rz, fmaf(Ry, Ry, Rx * Rx));
    const float rinv = rsqrt_approx(r2);   // |R| >= 1 cell half-width: normal, positive
    const float rinv2 = rinv * rinv;
    D[0] = rinv;
#pragma unroll
    for (int n = 1; n < P; ++n) {
        const float c1 = -(2.0f * n - 1.0f) / n;
        const float c2 = -(n - 1.0f) / n;
#pragma unroll
        for (int a = n; a >= 0; --a)
#pragma unroll
            for (int b = n - a; b >= 0; --b) {
                const int c = n - a - b;
                float s1 = 0.0f, s2 = 0.0f;
                if (a > 0) s1 = fmaf((float)a * Rx, D[MI<P>::idx(a - 1, b, c)], s1);
                if (b > 0) s1 = fmaf((float)b * Ry, D[MI<P>::idx(a, b - 1, c)], s1);
                if (c > 0) s1 = fmaf((float)c * Rz, D[MI<P>::idx(a, b, c - 1)], s1);
                if (a > 1) s2 = fmaf((float)(a * (a - 1)), D[MI<P>::idx(a - 2, b, c)], s2);
                if (b > 1) s2 = fmaf((float)(b * (b - 1)), D[MI<P>::idx(a, b - 2, c)], s2);
                if (c > 1) s2 = fmaf((float)(c * (c - 1)), D[MI<P>::idx(a, b, c - 2)], s2);
                D[MI<P>::idx(a, b, c)] = fmaf(c1, s1, c2 * s2) * rinv2;
            }
    }
}

// acc[idx(n) - N0] += sum_{|k| <= P-1-|n|} rho^|k| M[idx(k)] D[idx(n+k)] for the
// outputs with N0 <= idx(n) < N1; M is read from global memory (float4-aligned,
// TP floats) while the contraction runs, so only D and the accumulators of
// this output range stay in registers.
template <int P, int N0, int N1>
__device__ __forceinline__ void m2l_contract_range(const float4 *M4, const float *rho_pow, const float *D, float *acc)
{
    float4 m4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int nk = 0; nk < P; ++nk)
#pragma unroll
        for (int ka = nk; ka >= 0; --ka)
#pragma unroll
            for (int kb = nk - ka; kb >= 0; --kb) {
                const int kc = nk - ka - kb;
                const int ik = MI<P>::idx(ka, kb, kc);
                if ((ik & 3) == 0) m4 = __ldg(M4 + (ik >> 2));
                const float mraw = (ik & 3) == 0 ? m4.x : (ik & 3) == 1 ? m4.y : (ik & 3) == 2 ? m4.z : m4.w;
                const float m = mraw * rho_pow[nk];
#pragma unroll
                for (int nn = 0; nn + nk < P; ++nn)
#pragma unroll
                    for (int na = nn; na >= 0; --na)
#pragma unroll
                        for (int nb = nn - na; nb >= 0; --nb) {
                            const int nc = nn - na - nb;
                            const int in = MI<P>::idx(na, nb, nc);
                            if (in >= N0 && in < N1)
                                acc[in - N0] = fmaf(m, D[MI<P>::idx(na + ka, nb + kb, nc + kc)], acc[in - N0]);
                        }
            }
}

}  // namespace fmm
