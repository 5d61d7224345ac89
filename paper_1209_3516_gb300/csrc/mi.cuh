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

// ---------------------------------------------------------------------------
// Harmonic reduction of the M2L contraction.
// The derivatives of 1/|R| are harmonic in their index: D_{m+2e_x} + D_{m+2e_y}
// + D_{m+2e_z} = 0 (Laplace's equation).  Hence
//   - in sum_{|k|=e} M_k D_{n+k} every k with k_z >= 2 can be moved onto
//     k - 2e_z + 2e_x and k - 2e_z + 2e_y with the opposite sign: folding the
//     multipole once per cell onto its components with k_z <= 1 (2e + 1 per
//     degree e) leaves every contraction unchanged;
//   - the truncated local expansion L_n = sum_{|k| <= P-1-|n|} M_k D_{n+k} is
//     itself traceless (the three terms of L_{n+2e_x} + L_{n+2e_y} + L_{n+2e_z}
//     share one truncation), so only the outputs with n_z <= 1 are contracted
//     and L_n, n_z >= 2, follows as -L_{n-2e_z+2e_x} - L_{n-2e_z+2e_y};
//   - only D_m with m_z <= 2 is then needed: those with m_z <= 1 from the
//     recurrence below, which closes on that set, the rest from the same identity.
// At P = 8 a pair costs 876 multiply-adds and 85 derivatives instead of 1716
// and 120: the same truncated contraction, exact up to rounding.
template <int P> struct HI {
    static constexpr int F = P * P;   // components with c <= 1 and degree < P: sum (2e + 1)
    // (a, b, c <= 1), e = a + b + c: by degree, then c, then a descending
    __host__ __device__ static constexpr int fidx(int a, int b, int c)
    {
        return (a + b + c) * (a + b + c) + (c == 0 ? b : (a + b + 2) + b);
    }
    // derivatives with c <= 2: 1, 3, then 3 d per degree d >= 2
    __host__ __device__ static constexpr int doff(int d)
    {
        return d == 0 ? 0 : d == 1 ? 1 : 4 + 3 * (d * (d - 1) / 2 - 1);
    }
    __host__ __device__ static constexpr int didx(int a, int b, int c)
    {
        return doff(a + b + c) + (c == 0 ? b : c == 1 ? (a + b + 2) + b : (2 * (a + b + 2) + 1) + b);
    }
    static constexpr int ND = doff(P);
};

// D[didx(m)] = d^m (1/|R|) / dR^m for |m| <= P-1, m_z <= 2 (raw Cartesian
// derivatives).  The components with m_z <= 1 follow the recurrence (the
// Taylor-coefficient recurrence of Lindsay & Krasny, J. Comput. Phys. 172
// (2001), multiplied by m!)
//   |m| r^2 D_m = -(2|m|-1) sum_i m_i R_i D_{m-e_i} - (|m|-1) sum_i m_i (m_i-1) D_{m-2e_i},
// which lowers one index at a time and so closes on m_z <= 1; those with
// m_z = 2 then follow from the trace identity, D_{(a,b,2)} = -D_{(a+2,b,0)} - D_{(a,b+2,0)}.
template <int P>
__device__ __forceinline__ void laplace_derivatives_z2(float Rx, float Ry, float Rz, float *D)
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
        for (int c = 0; c <= 1; ++c)
#pragma unroll
            for (int a = n - c; a >= 0; --a) {
                if (c > n) continue;
                const int b = n - a - c;
                float s1 = 0.0f, s2 = 0.0f;
                if (a > 0) s1 = fmaf((float)a * Rx, D[HI<P>::didx(a - 1, b, c)], s1);
                if (b > 0) s1 = fmaf((float)b * Ry, D[HI<P>::didx(a, b - 1, c)], s1);
                if (c > 0) s1 = fmaf((float)c * Rz, D[HI<P>::didx(a, b, c - 1)], s1);
                if (a > 1) s2 = fmaf((float)(a * (a - 1)), D[HI<P>::didx(a - 2, b, c)], s2);
                if (b > 1) s2 = fmaf((float)(b * (b - 1)), D[HI<P>::didx(a, b - 2, c)], s2);
                D[HI<P>::didx(a, b, c)] = fmaf(c1, s1, c2 * s2) * rinv2;
            }
#pragma unroll
        for (int a = n - 2; a >= 0; --a) {
            const int b = n - 2 - a;
            D[HI<P>::didx(a, b, 2)] = -D[HI<P>::didx(a + 2, b, 0)] - D[HI<P>::didx(a, b + 2, 0)];
        }
    }
}

// acc[fidx(n)] += sum_{|k| <= P-1-|n|, k_z <= 1} rho^|k| Mf[fidx(k)] D[didx(n+k)]
// for the outputs with n_z <= 1; Mf4 is the folded multipole (F floats,
// float4-aligned; the caller stages it in shared memory).
template <int P>
__device__ __forceinline__ void m2l_contract_harmonic(const float4 *Mf4, const float *rho_pow, const float *D,
                                                      float *acc)
{
    float4 m4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int e = 0; e < P; ++e)
#pragma unroll
        for (int kc = 0; kc <= 1; ++kc)
#pragma unroll
            for (int ka = e - kc; ka >= 0; --ka) {
                if (kc > e) continue;
                const int kb = e - kc - ka;
                const int ik = HI<P>::fidx(ka, kb, kc);
                if ((ik & 3) == 0) m4 = Mf4[ik >> 2];
                const float mraw = (ik & 3) == 0 ? m4.x : (ik & 3) == 1 ? m4.y : (ik & 3) == 2 ? m4.z : m4.w;
                const float m = mraw * rho_pow[e];
#pragma unroll
                for (int d = 0; d + e < P; ++d)
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
}

}  // namespace fmm
