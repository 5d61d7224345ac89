/*
 * fmm_oracle.c -- CPU oracle for the dual-tree-traversal FMM of
 * R. Yokota, "An FMM Based on Dual Tree Traversal for Many-core
 * Architectures" (arXiv:1209.3516).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  The GPU library never
 * links, includes or calls it, and it shares no code, header, table or
 * constant generator with the GPU library.
 *
 * Plain, slow, obviously correct code: FP64 arithmetic everywhere, except the
 * three quantities that decide the interaction lists (cell radius, the MAC
 * distance and the MAC test), which are computed in FP32 with one rounding per
 * operation so that a list decision made here is the same decision an FP32
 * implementation makes.  Compile with -ffp-contract=off (no fused multiply-add)
 * and without -ffast-math.
 *
 * What is computed, with the passage of the paper it follows:
 *   - Laplace kernel: phi_i = sum_{j, r_ij != 0} q_j / r_ij and its gradient
 *     grad_i = -sum_j q_j (x_i - x_j) / r_ij^3 (Sec. 3.2, Table 3 caption:
 *     "Laplace kernel", potential and force).  No 1/(4 pi), no softening.
 *   - Octree of cubic cells addressed by 64-bit Morton keys, 21 levels
 *     (Table 2 "Morton key"; Sec. 2: a 64-bit key holds 21 levels), leaves of
 *     at most ncrit particles (Table 3 caption, N_crit).
 *   - Centre of expansion = geometric centre of the cell (Table 2), cell
 *     size for the MAC = tight radius B = max distance from that centre to the
 *     cell's particles (Sec. 3.2, B_max / R_max MAC).
 *   - MAC: a pair (A, B) is well separated when theta * |X_A - X_B| >
 *     B_A + B_B, i.e. (B_A + B_B) / R < theta, the bound whose leading error
 *     term is ((B_A + B_B) / R)^p (Sec. 3.2).
 *   - Dual tree traversal: Algorithm 3 (stack of cell pairs, split the larger
 *     cell) with Algorithm 4 (both leaves -> P2P, else MAC -> M2L, else push).
 *   - Cartesian Taylor expansions of order P (Sec. 3.1, Table 1): multipole
 *     and local coefficients for all multi-indices |k| <= P-1, M2L truncated at
 *     |n| + |k| <= P-1; operators P2M, M2M, M2L, L2L, L2P named in Sec. 3.2.
 *
 * Readings of points the paper leaves open (normalisation constants, the
 * split tie-break, the degree convention, coincident points) are stated at
 * the function that takes them.
 *
 * Adjoint (not in the paper: the derivatives of the sums above).  For a
 * scalar loss with upstream gradients a_i = dL/dphi_i and b_i = dL/dgrad_i,
 *   dq_k = Psi(x_k),  Psi(x) = sum_i a_i G(x - x_i) + sum_i b_i . grad_y G(x - y)|_{y = x_i}
 *   dx_k = a_k grad_k + H(x_k) b_k + q_k grad Psi(x_k),
 * with G = 1/r and H the Hessian of phi: Psi is the field of charges a and
 * dipoles b, so the same traversal lists, the same translation operators and a
 * dipole P2M give it; H b needs the second derivatives of the local expansion
 * of phi and of the P2P kernel.  orc_direct_backward is the plain definition
 * (O(N^2)); orc_backward takes these FMM steps.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_LEVELS 21          /* deepest level: 3 * 21 = 63 key bits */
#define ORC_MAXP 12            /* largest expansion order accepted */

/* ------------------------------------------------------------------ */
/* Multi-indices k = (kx, ky, kz) with |k| <= P-1, graded order.       */
/* ------------------------------------------------------------------ */

typedef struct {
    int t, u, j;                /* output index, input index, index of the summed multi-index */
    double coef;                /* constant factor of the term */
} orc_term;

typedef struct {
    int P;
    int nterms;                 /* P (P+1) (P+2) / 6 */
    int k[400][3];              /* enough for ORC_MAXP = 12 (364 terms) */
    int lookup[ORC_MAXP][ORC_MAXP][ORC_MAXP];  /* index of (kx,ky,kz), -1 if |k| > P-1 */
    /* term lists of the translation operators, built from their definitions */
    orc_term *m2l, *m2m, *l2l;
    int nm2l, nm2m, nl2l;
} orc_mindex;

static double orc_fact[2 * ORC_MAXP + 2];

static void orc_init_fact(void)
{
    orc_fact[0] = 1.0;
    for (int i = 1; i < 2 * ORC_MAXP + 2; ++i) orc_fact[i] = orc_fact[i - 1] * i;
}

static void orc_mindex_init(orc_mindex *mi, int P)
{
    orc_init_fact();
    mi->P = P;
    int t = 0;
    for (int a = 0; a < ORC_MAXP; ++a)
        for (int b = 0; b < ORC_MAXP; ++b)
            for (int c = 0; c < ORC_MAXP; ++c) mi->lookup[a][b][c] = -1;
    for (int deg = 0; deg < P; ++deg)
        for (int kx = deg; kx >= 0; --kx)
            for (int ky = deg - kx; ky >= 0; --ky) {
                int kz = deg - kx - ky;
                mi->k[t][0] = kx;
                mi->k[t][1] = ky;
                mi->k[t][2] = kz;
                mi->lookup[kx][ky][kz] = t;
                ++t;
            }
    mi->nterms = t;
    mi->m2l = mi->m2m = mi->l2l = NULL;
    mi->nm2l = mi->nm2m = mi->nl2l = 0;
}

static int orc_idx(const orc_mindex *mi, int kx, int ky, int kz)
{
    if (kx < 0 || ky < 0 || kz < 0) return -1;
    if (kx + ky + kz > mi->P - 1) return -1;
    return mi->lookup[kx][ky][kz];
}

/* k! = kx! ky! kz! */
static double orc_mfact(const int *k)
{
    return orc_fact[k[0]] * orc_fact[k[1]] * orc_fact[k[2]];
}

/* d^k = dx^kx dy^ky dz^kz */
static double orc_mpow(const double *d, const int *k)
{
    double r = 1.0;
    for (int a = 0; a < 3; ++a)
        for (int e = 0; e < k[a]; ++e) r *= d[a];
    return r;
}

/*
 * Term lists of M2L, M2M and L2L.  Each entry is one term of the operator's
 * sum as written at the operator below; building the list once only saves
 * recomputing the constant factors per call.
 */
static int orc_mindex_terms(orc_mindex *mi)
{
    int T = mi->nterms;
    mi->m2l = (orc_term *)malloc((size_t)T * T * sizeof(orc_term));
    mi->m2m = (orc_term *)malloc((size_t)T * T * sizeof(orc_term));
    mi->l2l = (orc_term *)malloc((size_t)T * T * sizeof(orc_term));
    if (!mi->m2l || !mi->m2m || !mi->l2l) return -1;
    for (int t = 0; t < T; ++t) {
        const int *a = mi->k[t];
        for (int u = 0; u < T; ++u) {
            const int *b = mi->k[u];
            int s[3] = {a[0] + b[0], a[1] + b[1], a[2] + b[2]};
            int d[3] = {a[0] - b[0], a[1] - b[1], a[2] - b[2]};
            int js = orc_idx(mi, s[0], s[1], s[2]);
            if (js >= 0) {
                /* M2L: output n = a, input k = b, derivative index n + k */
                double sign = ((b[0] + b[1] + b[2]) & 1) ? -1.0 : 1.0;
                orc_term e = {t, u, js, sign * orc_mfact(s) / orc_mfact(a)};
                mi->m2l[mi->nm2l++] = e;
                /* L2L: output k = a, shift m = b, input k + m */
                orc_term g = {t, u, js, orc_mfact(s) / (orc_mfact(a) * orc_mfact(b))};
                mi->l2l[mi->nl2l++] = g;
            }
            if (d[0] >= 0 && d[1] >= 0 && d[2] >= 0) {
                /* M2M: output k = a, input m = b, shift power k - m */
                int jd = orc_idx(mi, d[0], d[1], d[2]);
                orc_term e = {t, u, jd, 1.0 / orc_mfact(d)};
                mi->m2m[mi->nm2m++] = e;
            }
        }
    }
    return 0;
}

static void orc_mindex_free(orc_mindex *mi)
{
    free(mi->m2l); free(mi->m2m); free(mi->l2l);
    mi->m2l = mi->m2m = mi->l2l = NULL;
}

/* All monomials d^k for |k| <= P-1, in multi-index order. */
static void orc_monomials(const orc_mindex *mi, const double *d, double *w)
{
    for (int t = 0; t < mi->nterms; ++t) w[t] = orc_mpow(d, mi->k[t]);
}

int orc_nterms(int P) { return P * (P + 1) * (P + 2) / 6; }

/* The oracle's multi-index table, for tests that map coefficients. */
void orc_multi_indices(int P, int *k_out)
{
    if (P < 1 || P > ORC_MAXP) return;
    orc_mindex mi;
    orc_mindex_init(&mi, P);
    for (int t = 0; t < mi.nterms; ++t)
        for (int a = 0; a < 3; ++a) k_out[3 * t + a] = mi.k[t][a];
}

/* ------------------------------------------------------------------ */
/* Taylor coefficients of the Laplace kernel.                          */
/* ------------------------------------------------------------------ */

/*
 * b_m(R) = (1/m!) d^m/dR^m (1/|R|) for all |m| <= P-1 (Cartesian Taylor
 * expansion, Sec. 3.1).  The paper prints no formula; this uses the
 * published recurrence of Lindsay and Krasny (J. Comput. Phys. 172, 2001)
 * for the Taylor coefficients of 1/|R|:
 *   |m| |R|^2 b_m + (2|m| - 1) sum_i R_i b_{m - e_i} + (|m| - 1) sum_i b_{m - 2 e_i} = 0,
 * b_0 = 1/|R|, terms with a negative index component left out.
 */
static void orc_taylor_mi(const orc_mindex *mi, const double *R, double *b)
{
    double r2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
    b[0] = 1.0 / sqrt(r2);
    for (int t = 1; t < mi->nterms; ++t) {
        const int *m = mi->k[t];
        int deg = m[0] + m[1] + m[2];
        double s1 = 0.0, s2 = 0.0;
        for (int i = 0; i < 3; ++i) {
            int m1[3] = {m[0], m[1], m[2]};
            m1[i] -= 1;
            int j1 = orc_idx(mi, m1[0], m1[1], m1[2]);
            if (j1 >= 0) s1 += R[i] * b[j1];
            int m2[3] = {m[0], m[1], m[2]};
            m2[i] -= 2;
            int j2 = orc_idx(mi, m2[0], m2[1], m2[2]);
            if (j2 >= 0) s2 += b[j2];
        }
        b[t] = -((2.0 * deg - 1.0) * s1 + (deg - 1.0) * s2) / (deg * r2);
    }
}

void orc_taylor(int P, const double *R, double *b)
{
    if (P < 1 || P > ORC_MAXP) return;
    orc_mindex mi;
    orc_mindex_init(&mi, P);
    orc_taylor_mi(&mi, R, b);
}

/* ------------------------------------------------------------------ */
/* Expansion operators (Cartesian Taylor, all |k| <= P-1).             */
/* Multipole about the source centre X_S, local about the target       */
/* centre X_T; both stored as Taylor coefficients (1/k! folded in).    */
/* ------------------------------------------------------------------ */

/* P2M: M_k(C) += sum_j q_j d_j^k / k!, d_j = y_j - X_C. */
static void orc_p2m_mi(const orc_mindex *mi, int n, const double *y, const double *q,
                       const double *X, double *M)
{
    for (int j = 0; j < n; ++j) {
        double d[3] = {y[3 * j] - X[0], y[3 * j + 1] - X[1], y[3 * j + 2] - X[2]};
        for (int t = 0; t < mi->nterms; ++t)
            M[t] += q[j] * orc_mpow(d, mi->k[t]) / orc_mfact(mi->k[t]);
    }
}

/* M2M: M_k(P) += sum_{m <= k} M_m(C) delta^(k-m) / (k-m)!, delta = X_C - X_P. */
static void orc_m2m_mi(const orc_mindex *mi, const double *Mc, const double *Xc,
                       const double *Xp, double *Mp)
{
    double delta[3] = {Xc[0] - Xp[0], Xc[1] - Xp[1], Xc[2] - Xp[2]};
    double w[400];
    orc_monomials(mi, delta, w);
    for (int e = 0; e < mi->nm2m; ++e) {
        const orc_term *tm = &mi->m2m[e];
        Mp[tm->t] += Mc[tm->u] * w[tm->j] * tm->coef;
    }
}

/*
 * M2L: with the multipole expanded about X_S (kernel G(x - y), source offset
 * -d) and the local about X_T,
 *   L_n(T) += sum_{|k| <= P-1-|n|} (-1)^|k| M_k(S) ((n+k)! / n!) b_{n+k}(X_T - X_S).
 * Degree convention (the paper only fixes the error as ((B_A+B_B)/R)^p):
 * the first neglected total degree |n| + |k| is P.
 */
static void orc_m2l_mi(const orc_mindex *mi, const double *M, const double *Xs,
                       const double *Xt, double *L)
{
    double R[3] = {Xt[0] - Xs[0], Xt[1] - Xs[1], Xt[2] - Xs[2]};
    double b[400];
    orc_taylor_mi(mi, R, b);
    for (int e = 0; e < mi->nm2l; ++e) {
        const orc_term *tm = &mi->m2l[e];
        L[tm->t] += tm->coef * M[tm->u] * b[tm->j];
    }
}

/* L2L: L_k(C) += sum_m L_{k+m}(P) ((k+m)! / (k! m!)) d^m, d = X_C - X_P. */
static void orc_l2l_mi(const orc_mindex *mi, const double *Lp, const double *Xp,
                       const double *Xc, double *Lc)
{
    double d[3] = {Xc[0] - Xp[0], Xc[1] - Xp[1], Xc[2] - Xp[2]};
    double w[400];
    orc_monomials(mi, d, w);
    for (int e = 0; e < mi->nl2l; ++e) {
        const orc_term *tm = &mi->l2l[e];
        Lc[tm->t] += Lp[tm->j] * tm->coef * w[tm->u];
    }
}

/* L2P: phi += sum_n L_n r^n, grad_a += sum_n L_n n_a r^(n - e_a), r = x - X_T. */
static void orc_l2p_mi(const orc_mindex *mi, const double *L, const double *Xt, int n,
                       const double *x, double *phi, double *grad)
{
    for (int i = 0; i < n; ++i) {
        double r[3] = {x[3 * i] - Xt[0], x[3 * i + 1] - Xt[1], x[3 * i + 2] - Xt[2]};
        double p = 0.0, g[3] = {0.0, 0.0, 0.0};
        for (int t = 0; t < mi->nterms; ++t) {
            const int *k = mi->k[t];
            p += L[t] * orc_mpow(r, k);
            for (int a = 0; a < 3; ++a) {
                if (k[a] == 0) continue;
                int km[3] = {k[0], k[1], k[2]};
                km[a] -= 1;
                g[a] += L[t] * k[a] * orc_mpow(r, km);
            }
        }
        phi[i] += p;
        for (int a = 0; a < 3; ++a) grad[3 * i + a] += g[a];
    }
}

/*
 * Dipole P2M: the multipole of a dipole p at y is p . grad_y of the multipole
 * of a unit charge at y: d/dy_c (d^k / k!) = d^(k - e_c) / (k - e_c)!, so
 *   M_k(C) += a_j d_j^k / k! + sum_c p_{j,c} d_j^(k - e_c) / (k - e_c)!,  d_j = y_j - X_C,
 * for sources carrying a charge a_j and a dipole p_j (3 per source).
 */
static void orc_p2m_dipole_mi(const orc_mindex *mi, int n, const double *y, const double *a,
                              const double *p, const double *X, double *M)
{
    for (int j = 0; j < n; ++j) {
        double d[3] = {y[3 * j] - X[0], y[3 * j + 1] - X[1], y[3 * j + 2] - X[2]};
        for (int t = 0; t < mi->nterms; ++t) {
            const int *k = mi->k[t];
            M[t] += a[j] * orc_mpow(d, k) / orc_mfact(k);
            for (int c = 0; c < 3; ++c) {
                if (k[c] == 0) continue;
                int km[3] = {k[0], k[1], k[2]};
                km[c] -= 1;
                M[t] += p[3 * j + c] * orc_mpow(d, km) / orc_mfact(km);
            }
        }
    }
}

/*
 * Hessian-vector product of a local expansion: hv_a += sum_b v_b d^2/dx_a dx_b
 * sum_n L_n r^n, r = x - X_T, for one point x and one vector v.
 */
static void orc_l2p_hess_mi(const orc_mindex *mi, const double *L, const double *Xt,
                            const double *x, const double *v, double *hv)
{
    double r[3] = {x[0] - Xt[0], x[1] - Xt[1], x[2] - Xt[2]};
    for (int t = 0; t < mi->nterms; ++t) {
        const int *k = mi->k[t];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                /* d/dx_b d/dx_a r^k: factor k_a (k_b - [a == b]) times r^(k - e_a - e_b) */
                int km[3] = {k[0], k[1], k[2]};
                double f = km[a];
                km[a] -= 1;
                if (f == 0.0) continue;
                f *= km[b];
                km[b] -= 1;
                if (f == 0.0) continue;
                hv[a] += L[t] * f * orc_mpow(r, km) * v[b];
            }
    }
}

/* Stand-alone operator entry points (arrays in the oracle's multi-index order). */
static orc_mindex *orc_mindex_new(int P)
{
    if (P < 1 || P > ORC_MAXP) return NULL;
    orc_mindex *mi = (orc_mindex *)malloc(sizeof(orc_mindex));
    if (!mi) return NULL;
    orc_mindex_init(mi, P);
    if (orc_mindex_terms(mi)) { orc_mindex_free(mi); free(mi); return NULL; }
    return mi;
}

static void orc_mindex_delete(orc_mindex *mi)
{
    if (!mi) return;
    orc_mindex_free(mi);
    free(mi);
}

int orc_p2m(int P, int n, const double *y, const double *q, const double *X, double *M)
{
    orc_mindex *mi = orc_mindex_new(P);
    if (!mi) return -1;
    orc_p2m_mi(mi, n, y, q, X, M);
    orc_mindex_delete(mi);
    return 0;
}

int orc_m2m(int P, const double *Mc, const double *Xc, const double *Xp, double *Mp)
{
    orc_mindex *mi = orc_mindex_new(P);
    if (!mi) return -1;
    orc_m2m_mi(mi, Mc, Xc, Xp, Mp);
    orc_mindex_delete(mi);
    return 0;
}

int orc_m2l(int P, const double *M, const double *Xs, const double *Xt, double *L)
{
    orc_mindex *mi = orc_mindex_new(P);
    if (!mi) return -1;
    orc_m2l_mi(mi, M, Xs, Xt, L);
    orc_mindex_delete(mi);
    return 0;
}

int orc_l2l(int P, const double *Lp, const double *Xp, const double *Xc, double *Lc)
{
    orc_mindex *mi = orc_mindex_new(P);
    if (!mi) return -1;
    orc_l2l_mi(mi, Lp, Xp, Xc, Lc);
    orc_mindex_delete(mi);
    return 0;
}

int orc_l2p(int P, const double *L, const double *Xt, int n, const double *x, double *phi,
            double *grad)
{
    orc_mindex *mi = orc_mindex_new(P);
    if (!mi) return -1;
    orc_l2p_mi(mi, L, Xt, n, x, phi, grad);
    orc_mindex_delete(mi);
    return 0;
}

int orc_p2m_dipole(int P, int n, const double *y, const double *a, const double *p, const double *X,
                   double *M)
{
    orc_mindex *mi = orc_mindex_new(P);
    if (!mi) return -1;
    orc_p2m_dipole_mi(mi, n, y, a, p, X, M);
    orc_mindex_delete(mi);
    return 0;
}

int orc_l2p_hess(int P, const double *L, const double *Xt, const double *x, const double *v, double *hv)
{
    orc_mindex *mi = orc_mindex_new(P);
    if (!mi) return -1;
    orc_l2p_hess_mi(mi, L, Xt, x, v, hv);
    orc_mindex_delete(mi);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Direct O(N^2) sum: the plain definition the FMM approximates.       */
/* ------------------------------------------------------------------ */

/*
 * phi_i = sum_{j: r_ij != 0} q_j / r_ij, grad_i = -sum_j q_j (x_i - x_j) / r_ij^3,
 * in FP64 on the caller's coordinates.  A pair at distance 0 (including
 * i = j) contributes nothing (the paper is silent on coincident points).
 * targets == NULL: all N targets, outputs of length N; otherwise outputs of
 * length nt for the listed target indices.
 */
void orc_direct(int64_t N, const double *x, const double *q, int64_t nt, const int64_t *targets,
                double *phi, double *grad)
{
    int64_t nout = targets ? nt : N;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nout; ++t) {
        int64_t i = targets ? targets[t] : t;
        double p = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int64_t j = 0; j < N; ++j) {
            double dx = x[3 * i] - x[3 * j];
            double dy = x[3 * i + 1] - x[3 * j + 1];
            double dz = x[3 * i + 2] - x[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            p += q[j] / r;
            double w = q[j] / (r2 * r);
            gx -= w * dx;
            gy -= w * dy;
            gz -= w * dz;
        }
        phi[t] = p;
        grad[3 * t] = gx;
        grad[3 * t + 1] = gy;
        grad[3 * t + 2] = gz;
    }
}

/*
 * Adjoint of the direct sum, written out from the definition.  With
 * phi_i = sum_{j != i} q_j / r_ij and grad_i = -sum_{j != i} q_j d_ij / r_ij^3
 * (d_ij = x_i - x_j), and upstream gradients a_i (potential) and b_i
 * (gradient, 3 per particle) of a scalar loss L:
 *   dL/dq_k = sum_{i != k} [ a_i / r_ik - b_i . d_ik / r_ik^3 ]
 *   dL/dx_k = a_k grad_k + sum_{i != k} a_i q_k d_ik / r_ik^3
 *           + sum_{j != k} q_j H(d_kj) b_k - sum_{i != k} q_k H(d_ik) b_i,
 * H(d) = -I / r^3 + 3 d d^T / r^5 (the Hessian of 1/|d|).  Pairs at distance
 * 0 contribute nothing, as in the forward sum.  a or b may be NULL (zero).
 * targets == NULL: all N outputs; otherwise the nt listed indices.
 */
void orc_direct_backward(int64_t N, const double *x, const double *q, const double *a,
                         const double *b, int64_t nt, const int64_t *targets, double *dq,
                         double *dx)
{
    int64_t nout = targets ? nt : N;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nout; ++t) {
        int64_t k = targets ? targets[t] : t;
        double g[3] = {0.0, 0.0, 0.0}, s_dq = 0.0, s_dx[3] = {0.0, 0.0, 0.0};
        double bk[3] = {0.0, 0.0, 0.0};
        if (b) for (int c = 0; c < 3; ++c) bk[c] = b[3 * k + c];
        for (int64_t i = 0; i < N; ++i) {
            double d[3];  /* d_ik = x_i - x_k */
            for (int c = 0; c < 3; ++c) d[c] = x[3 * i + c] - x[3 * k + c];
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (r2 == 0.0) continue;
            double r = sqrt(r2), r3 = r2 * r, r5 = r3 * r2;
            double ai = a ? a[i] : 0.0;
            double bi[3] = {0.0, 0.0, 0.0};
            if (b) for (int c = 0; c < 3; ++c) bi[c] = b[3 * i + c];
            /* potential and gradient at k (d_ki = -d_ik) */
            for (int c = 0; c < 3; ++c) g[c] += q[i] * d[c] / r3;
            /* dq_k */
            s_dq += ai / r - (bi[0] * d[0] + bi[1] * d[1] + bi[2] * d[2]) / r3;
            /* dx_k: a_i q_k d_ik / r^3 */
            for (int c = 0; c < 3; ++c) s_dx[c] += ai * q[k] * d[c] / r3;
            /* q_i H(d_ki) b_k - q_k H(d_ik) b_i; H is even in d */
            double dbk = d[0] * bk[0] + d[1] * bk[1] + d[2] * bk[2];
            double dbi = d[0] * bi[0] + d[1] * bi[1] + d[2] * bi[2];
            for (int c = 0; c < 3; ++c) {
                double Hbk = -bk[c] / r3 + 3.0 * d[c] * dbk / r5;
                double Hbi = -bi[c] / r3 + 3.0 * d[c] * dbi / r5;
                s_dx[c] += q[i] * Hbk - q[k] * Hbi;
            }
        }
        double ak = a ? a[k] : 0.0;
        dq[t] = s_dq;
        for (int c = 0; c < 3; ++c) dx[3 * t + c] = ak * g[c] + s_dx[c];
    }
}

/* ------------------------------------------------------------------ */
/* Tree, traversal and FMM evaluation.                                 */
/* ------------------------------------------------------------------ */

typedef struct {
    int64_t a, b;
} orc_pair;

typedef struct {
    orc_pair *v;
    int64_t n, cap;
} orc_pairvec;

static int orc_pv_push(orc_pairvec *pv, int64_t a, int64_t b)
{
    if (pv->n == pv->cap) {
        int64_t nc = pv->cap ? 2 * pv->cap : 1024;
        orc_pair *nv = (orc_pair *)realloc(pv->v, (size_t)nc * sizeof(orc_pair));
        if (!nv) return -1;
        pv->v = nv;
        pv->cap = nc;
    }
    pv->v[pv->n].a = a;
    pv->v[pv->n].b = b;
    pv->n++;
    return 0;
}

typedef struct orc_fmm {
    int64_t N;
    int P, ncrit;
    float theta;
    int64_t hybrid_min_pairs;   /* < 0: Algorithm 4 as printed; else the M2L / P2P hybrid (orc_interact) */
    orc_mindex mi;
    /* normalisation */
    double centre[3], h;
    /* particles in sorted (key, index) order */
    uint64_t *key;     /* sorted keys */
    int64_t *perm;     /* perm[s] = original index of sorted particle s */
    double *u;         /* normalised positions, FP64, N x 3 (sorted) */
    float *u32;        /* the same rounded to FP32 (geometry only) */
    /* cells in breadth-first order */
    int64_t ncells, cellcap;
    int *level;
    uint64_t *prefix;
    int64_t *pbeg, *pcnt, *cbeg, *parent;
    int *ccnt;
    float *cx;         /* centre, ncells x 3 */
    float *radius;
    /* interaction lists (cell indices) */
    orc_pairvec m2l, p2p;
    int built;
} orc_fmm;

static void orc_free_tree(orc_fmm *f)
{
    free(f->key); free(f->perm); free(f->u); free(f->u32);
    free(f->level); free(f->prefix); free(f->pbeg); free(f->pcnt); free(f->cbeg);
    free(f->parent); free(f->ccnt); free(f->cx); free(f->radius);
    free(f->m2l.v); free(f->p2p.v);
    f->key = NULL; f->perm = NULL; f->u = NULL; f->u32 = NULL;
    f->level = NULL; f->prefix = NULL; f->pbeg = NULL; f->pcnt = NULL; f->cbeg = NULL;
    f->parent = NULL; f->ccnt = NULL; f->cx = NULL; f->radius = NULL;
    memset(&f->m2l, 0, sizeof(f->m2l));
    memset(&f->p2p, 0, sizeof(f->p2p));
    f->ncells = f->cellcap = 0;
    f->built = 0;
}

orc_fmm *orc_create(int64_t N, int P, float theta, int ncrit)
{
    if (N < 1 || P < 1 || P > ORC_MAXP || ncrit < 1 || !(theta >= 0.0f)) return NULL;
    orc_fmm *f = (orc_fmm *)calloc(1, sizeof(orc_fmm));
    if (!f) return NULL;
    f->N = N;
    f->P = P;
    f->theta = theta;
    f->ncrit = ncrit;
    f->hybrid_min_pairs = -1;
    orc_mindex_init(&f->mi, P);
    if (orc_mindex_terms(&f->mi)) { orc_mindex_free(&f->mi); free(f); return NULL; }
    return f;
}

void orc_destroy(orc_fmm *f)
{
    if (!f) return;
    orc_free_tree(f);
    orc_mindex_free(&f->mi);
    free(f);
}

/* Morton interleave of three 21-bit integers: x at bit 3b, y at 3b+1, z at 3b+2. */
uint64_t orc_morton(uint32_t ix, uint32_t iy, uint32_t iz)
{
    uint64_t key = 0;
    for (int b = 0; b < ORC_LEVELS; ++b) {
        key |= (uint64_t)((ix >> b) & 1u) << (3 * b);
        key |= (uint64_t)((iy >> b) & 1u) << (3 * b + 1);
        key |= (uint64_t)((iz >> b) & 1u) << (3 * b + 2);
    }
    return key;
}

/* Inverse of orc_morton restricted to the low 3*nlev bits. */
static void orc_demorton(uint64_t key, int nlev, uint32_t *ix, uint32_t *iy, uint32_t *iz)
{
    uint32_t a = 0, b = 0, c = 0;
    for (int l = 0; l < nlev; ++l) {
        a |= (uint32_t)((key >> (3 * l)) & 1u) << l;
        b |= (uint32_t)((key >> (3 * l + 1)) & 1u) << l;
        c |= (uint32_t)((key >> (3 * l + 2)) & 1u) << l;
    }
    *ix = a; *iy = b; *iz = c;
}

/*
 * Normalisation to the cube (-1, 1)^3 and Morton keys.  The paper only says
 * keys are built from a global cube (Table 2, Sec. 2); the reading taken:
 *   c = (min + max) / 2 per dimension,  h = (max_d extent / 2) * (1 + 2^-20),
 *   h = 1 when every particle coincides,  u = (x - c) / h,
 *   i_d = min(floor((u_d + 1) * 2^20), 2^21 - 1),  key = interleave(i_x, i_y, i_z).
 * Each operation is one FP64 rounding, in that order.
 */
static int orc_normalise(orc_fmm *f, const double *x, double *u, uint64_t *key)
{
    int64_t N = f->N;
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = x[a]; hi[a] = x[a]; }
    for (int64_t i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = x[3 * i + a];
            if (!isfinite(v)) return -1;
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        f->centre[a] = (lo[a] + hi[a]) * 0.5;
        double e = hi[a] - lo[a];
        if (e > ext) ext = e;
    }
    double h = ext * 0.5;
    h = h * (1.0 + 0x1p-20);
    if (h == 0.0) h = 1.0;
    f->h = h;
    for (int64_t i = 0; i < N; ++i) {
        uint32_t ic[3];
        for (int a = 0; a < 3; ++a) {
            double v = (x[3 * i + a] - f->centre[a]) / h;
            u[3 * i + a] = v;
            double s = floor((v + 1.0) * 0x1p20);
            if (s < 0.0) s = 0.0;
            if (s > 2097151.0) s = 2097151.0;
            ic[a] = (uint32_t)s;
        }
        key[i] = orc_morton(ic[0], ic[1], ic[2]);
    }
    return 0;
}

typedef struct {
    uint64_t key;
    int64_t idx;
} orc_keyidx;

static int orc_cmp_keyidx(const void *pa, const void *pb)
{
    const orc_keyidx *a = (const orc_keyidx *)pa, *b = (const orc_keyidx *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->idx != b->idx) return a->idx < b->idx ? -1 : 1;
    return 0;
}

static int orc_cell_grow(orc_fmm *f)
{
    int64_t nc = f->cellcap ? 2 * f->cellcap : 1024;
#define ORC_GROW(ptr, T) do { T *q_ = (T *)realloc(f->ptr, (size_t)nc * sizeof(T)); if (!q_) return -1; f->ptr = q_; } while (0)
    ORC_GROW(level, int);
    ORC_GROW(prefix, uint64_t);
    ORC_GROW(pbeg, int64_t);
    ORC_GROW(pcnt, int64_t);
    ORC_GROW(cbeg, int64_t);
    ORC_GROW(parent, int64_t);
    ORC_GROW(ccnt, int);
#undef ORC_GROW
    f->cellcap = nc;
    return 0;
}

static int orc_cell_add(orc_fmm *f, int level, uint64_t prefix, int64_t pbeg, int64_t pcnt,
                        int64_t parent)
{
    if (f->ncells == f->cellcap && orc_cell_grow(f)) return -1;
    int64_t c = f->ncells++;
    f->level[c] = level;
    f->prefix[c] = prefix;
    f->pbeg[c] = pbeg;
    f->pcnt[c] = pcnt;
    f->cbeg[c] = 0;
    f->ccnt[c] = 0;
    f->parent[c] = parent;
    return 0;
}

static int orc_is_leaf(const orc_fmm *f, int64_t c) { return f->ccnt[c] == 0; }

/*
 * MAC in FP32, one rounding per operation (Sec. 3.2, "FMM MAC"):
 *   R = sqrt((dx*dx + dy*dy) + dz*dz), accept iff theta * R > B_A + B_B.
 * A cell paired with itself has R = 0 and is never accepted.
 */
static int orc_mac(const orc_fmm *f, int64_t A, int64_t B)
{
    float dx = f->cx[3 * A] - f->cx[3 * B];
    float dy = f->cx[3 * A + 1] - f->cx[3 * B + 1];
    float dz = f->cx[3 * A + 2] - f->cx[3 * B + 2];
    float xx = dx * dx;
    float yy = dy * dy;
    float zz = dz * dz;
    float r2 = xx + yy;
    r2 = r2 + zz;
    float R = sqrtf(r2);
    float lhs = f->theta * R;
    float rhs = f->radius[A] + f->radius[B];
    return lhs > rhs;
}

/* Algorithm 4, Interact(A, B). */
/*
 * Algorithm 4: both leaves -> P2P (checked before the MAC, as printed); else
 * MAC -> M2L; else push.  With hybrid_min_pairs >= 0 (the M2L / P2P hybrid
 * the paper describes for exaFMM, Sec. 2: the choice between the two kernels
 * at the leaves is tuned): a leaf pair that passes the MAC and holds at least
 * hybrid_min_pairs particle pairs (n_A n_B) is an M2L pair instead.
 */
static int orc_interact(orc_fmm *f, orc_pairvec *stack, int64_t A, int64_t B)
{
    if (orc_is_leaf(f, A) && orc_is_leaf(f, B)) {
        if (f->hybrid_min_pairs >= 0 && f->pcnt[A] * f->pcnt[B] >= f->hybrid_min_pairs && orc_mac(f, A, B))
            return orc_pv_push(&f->m2l, A, B);
        return orc_pv_push(&f->p2p, A, B);
    }
    if (orc_mac(f, A, B)) return orc_pv_push(&f->m2l, A, B);
    return orc_pv_push(stack, A, B);
}

/* The M2L / P2P hybrid for the next build: min_pairs < 0 turns it off. */
void orc_set_hybrid(orc_fmm *f, int64_t min_pairs) { f->hybrid_min_pairs = min_pairs; }

/*
 * Algorithm 3, dual tree traversal from the pair (root, root).
 * "Target cell is larger than source cell" is read as: split the target A
 * when B is a leaf, or when A is not a leaf and B_A > B_B; otherwise split
 * the source B (ties split the source).  A root that is itself a leaf gives
 * the single P2P pair (root, root).
 */
static int orc_traverse(orc_fmm *f)
{
    orc_pairvec stack = {0};
    f->m2l.n = 0;
    f->p2p.n = 0;
    if (orc_is_leaf(f, 0)) return orc_pv_push(&f->p2p, 0, 0);
    if (orc_pv_push(&stack, 0, 0)) return -1;
    while (stack.n > 0) {
        orc_pair pr = stack.v[--stack.n];
        int64_t A = pr.a, B = pr.b;
        int split_target = orc_is_leaf(f, B) || (!orc_is_leaf(f, A) && f->radius[A] > f->radius[B]);
        if (split_target) {
            for (int c = 0; c < f->ccnt[A]; ++c)
                if (orc_interact(f, &stack, f->cbeg[A] + c, B)) { free(stack.v); return -1; }
        } else {
            for (int c = 0; c < f->ccnt[B]; ++c)
                if (orc_interact(f, &stack, A, f->cbeg[B] + c)) { free(stack.v); return -1; }
        }
    }
    free(stack.v);
    return 0;
}

/*
 * Build: normalise, Morton keys, stable sort by (key, original index),
 * top-down octree (a cell with more than ncrit particles below level 21
 * splits into its non-empty octants, in key order), cell geometry, and the
 * dual tree traversal.  Returns 0, or -1 on non-finite input / no memory.
 */
int orc_build(orc_fmm *f, const double *x)
{
    int64_t N = f->N;
    orc_free_tree(f);
    double *u0 = (double *)malloc((size_t)N * 3 * sizeof(double));
    uint64_t *k0 = (uint64_t *)malloc((size_t)N * sizeof(uint64_t));
    orc_keyidx *ki = (orc_keyidx *)malloc((size_t)N * sizeof(orc_keyidx));
    f->key = (uint64_t *)malloc((size_t)N * sizeof(uint64_t));
    f->perm = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    f->u = (double *)malloc((size_t)N * 3 * sizeof(double));
    f->u32 = (float *)malloc((size_t)N * 3 * sizeof(float));
    if (!u0 || !k0 || !ki || !f->key || !f->perm || !f->u || !f->u32) goto fail;
    if (orc_normalise(f, x, u0, k0)) goto fail;
    for (int64_t i = 0; i < N; ++i) { ki[i].key = k0[i]; ki[i].idx = i; }
    qsort(ki, (size_t)N, sizeof(orc_keyidx), orc_cmp_keyidx);
    for (int64_t s = 0; s < N; ++s) {
        int64_t i = ki[s].idx;
        f->key[s] = ki[s].key;
        f->perm[s] = i;
        for (int a = 0; a < 3; ++a) {
            f->u[3 * s + a] = u0[3 * i + a];
            f->u32[3 * s + a] = (float)u0[3 * i + a];
        }
    }
    free(u0); u0 = NULL;
    free(k0); k0 = NULL;
    free(ki); ki = NULL;

    /* top-down octree, breadth first */
    if (orc_cell_add(f, 0, 0, 0, N, -1)) goto fail;
    for (int64_t c = 0; c < f->ncells; ++c) {
        if (f->pcnt[c] <= f->ncrit || f->level[c] >= ORC_LEVELS) continue;
        int cl = f->level[c] + 1;
        int shift = 3 * (ORC_LEVELS - cl);
        int64_t s = f->pbeg[c], e = f->pbeg[c] + f->pcnt[c];
        f->cbeg[c] = f->ncells;
        int nch = 0;
        for (int o = 0; o < 8; ++o) {
            uint64_t cp = (f->prefix[c] << 3) | (uint64_t)o;
            int64_t b = s;
            while (s < e && (f->key[s] >> shift) == cp) ++s;
            if (s > b) {
                if (orc_cell_add(f, cl, cp, b, s - b, c)) goto fail;
                ++nch;
            }
        }
        f->ccnt[c] = nch;
    }

    /* geometry: geometric centre (exact in FP32) and tight radius in FP32 */
    f->cx = (float *)malloc((size_t)f->ncells * 3 * sizeof(float));
    f->radius = (float *)malloc((size_t)f->ncells * sizeof(float));
    if (!f->cx || !f->radius) goto fail;
    for (int64_t c = 0; c < f->ncells; ++c) {
        uint32_t ic[3];
        int l = f->level[c];
        orc_demorton(f->prefix[c], l, &ic[0], &ic[1], &ic[2]);
        for (int a = 0; a < 3; ++a)
            f->cx[3 * c + a] = (float)((2.0 * ic[a] + 1.0) * ldexp(1.0, -l) - 1.0);
        float best = 0.0f;
        for (int64_t j = f->pbeg[c]; j < f->pbeg[c] + f->pcnt[c]; ++j) {
            float dx = f->u32[3 * j] - f->cx[3 * c];
            float dy = f->u32[3 * j + 1] - f->cx[3 * c + 1];
            float dz = f->u32[3 * j + 2] - f->cx[3 * c + 2];
            float xx = dx * dx;
            float yy = dy * dy;
            float zz = dz * dz;
            float r2 = xx + yy;
            r2 = r2 + zz;
            if (r2 > best) best = r2;
        }
        f->radius[c] = sqrtf(best);
    }

    if (orc_traverse(f)) goto fail;
    f->built = 1;
    return 0;
fail:
    free(u0); free(k0); free(ki);
    orc_free_tree(f);
    return -1;
}

static int orc_cmp_pair(const void *pa, const void *pb)
{
    const orc_pair *a = (const orc_pair *)pa, *b = (const orc_pair *)pb;
    if (a->a != b->a) return a->a < b->a ? -1 : 1;
    if (a->b != b->b) return a->b < b->b ? -1 : 1;
    return 0;
}

static void orc_centre_d(const orc_fmm *f, int64_t c, double *X)
{
    for (int a = 0; a < 3; ++a) X[a] = (double)f->cx[3 * c + a];
}

/*
 * Evaluation: P2M on leaves, M2M bottom-up, M2L over the list, L2L top-down,
 * L2P and P2P on leaves, back to the caller's order and units
 * (phi / h, grad / h^2: the kernel is homogeneous of degree -1).
 * targets == NULL evaluates all N particles; otherwise only the nt listed
 * original indices (outputs of length nt), computing just the local
 * expansions those targets need.
 */
int orc_evaluate(orc_fmm *f, const double *q, int64_t nt, const int64_t *targets, double *phi,
                 double *grad)
{
    if (!f->built) return -1;
    const orc_mindex *mi = &f->mi;
    int T = mi->nterms;
    int64_t N = f->N, nc = f->ncells;
    double *qs = (double *)malloc((size_t)N * sizeof(double));
    double *M = (double *)calloc((size_t)nc * T, sizeof(double));
    double *L = (double *)calloc((size_t)nc * T, sizeof(double));
    double *ps = (double *)calloc((size_t)N, sizeof(double));
    double *gs = (double *)calloc((size_t)N * 3, sizeof(double));
    char *want = (char *)calloc((size_t)N, 1);      /* sorted particle wanted */
    char *need = (char *)calloc((size_t)nc, 1);     /* cell's local expansion needed */
    int64_t *inv = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    orc_pair *m2l = NULL, *p2p = NULL;
    int64_t *m2l_off = NULL, *p2p_off = NULL;
    int rc = -1;
    if (!qs || !M || !L || !ps || !gs || !want || !need || !inv) goto done;
    for (int64_t s = 0; s < N; ++s) { qs[s] = q[f->perm[s]]; inv[f->perm[s]] = s; }
    if (targets) {
        for (int64_t t = 0; t < nt; ++t) {
            if (targets[t] < 0 || targets[t] >= N) goto done;
            want[inv[targets[t]]] = 1;
        }
    } else {
        memset(want, 1, (size_t)N);
    }
    /* cells whose local expansion is needed: leaves holding a wanted particle and their ancestors */
    for (int64_t c = nc - 1; c >= 0; --c) {
        if (orc_is_leaf(f, c)) {
            for (int64_t j = f->pbeg[c]; j < f->pbeg[c] + f->pcnt[c]; ++j)
                if (want[j]) { need[c] = 1; break; }
        }
        if (need[c] && f->parent[c] >= 0) need[f->parent[c]] = 1;
    }

    /* upward pass */
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < nc; ++c) {
        if (!orc_is_leaf(f, c)) continue;
        double X[3];
        orc_centre_d(f, c, X);
        orc_p2m_mi(mi, (int)f->pcnt[c], f->u + 3 * f->pbeg[c], qs + f->pbeg[c], X, M + c * T);
    }
    for (int64_t c = nc - 1; c >= 1; --c) {
        double Xc[3], Xp[3];
        int64_t p = f->parent[c];
        orc_centre_d(f, c, Xc);
        orc_centre_d(f, p, Xp);
        orc_m2m_mi(mi, M + c * T, Xc, Xp, M + p * T);
    }

    /* M2L, grouped by target so each target is written by one thread */
    m2l = (orc_pair *)malloc((size_t)(f->m2l.n + 1) * sizeof(orc_pair));
    m2l_off = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    if (!m2l || !m2l_off) goto done;
    memcpy(m2l, f->m2l.v, (size_t)f->m2l.n * sizeof(orc_pair));
    qsort(m2l, (size_t)f->m2l.n, sizeof(orc_pair), orc_cmp_pair);
    for (int64_t e = 0; e < f->m2l.n; ++e) m2l_off[m2l[e].a + 1]++;
    for (int64_t c = 0; c < nc; ++c) m2l_off[c + 1] += m2l_off[c];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < nc; ++c) {
        if (!need[c]) continue;
        double Xt[3];
        orc_centre_d(f, c, Xt);
        for (int64_t e = m2l_off[c]; e < m2l_off[c + 1]; ++e) {
            double Xs[3];
            int64_t s = m2l[e].b;
            orc_centre_d(f, s, Xs);
            orc_m2l_mi(mi, M + s * T, Xs, Xt, L + c * T);
        }
    }

    /* downward pass */
    for (int64_t c = 1; c < nc; ++c) {
        if (!need[c]) continue;
        double Xc[3], Xp[3];
        int64_t p = f->parent[c];
        orc_centre_d(f, c, Xc);
        orc_centre_d(f, p, Xp);
        orc_l2l_mi(mi, L + p * T, Xp, Xc, L + c * T);
    }

    /* L2P and P2P on wanted particles, grouped by target leaf */
    p2p = (orc_pair *)malloc((size_t)(f->p2p.n + 1) * sizeof(orc_pair));
    p2p_off = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    if (!p2p || !p2p_off) goto done;
    memcpy(p2p, f->p2p.v, (size_t)f->p2p.n * sizeof(orc_pair));
    qsort(p2p, (size_t)f->p2p.n, sizeof(orc_pair), orc_cmp_pair);
    for (int64_t e = 0; e < f->p2p.n; ++e) p2p_off[p2p[e].a + 1]++;
    for (int64_t c = 0; c < nc; ++c) p2p_off[c + 1] += p2p_off[c];
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < nc; ++c) {
        if (!orc_is_leaf(f, c) || !need[c]) continue;
        double Xt[3];
        orc_centre_d(f, c, Xt);
        for (int64_t i = f->pbeg[c]; i < f->pbeg[c] + f->pcnt[c]; ++i) {
            if (!want[i]) continue;
            orc_l2p_mi(mi, L + c * T, Xt, 1, f->u + 3 * i, ps + i, gs + 3 * i);
            for (int64_t e = p2p_off[c]; e < p2p_off[c + 1]; ++e) {
                int64_t s = p2p[e].b;
                for (int64_t j = f->pbeg[s]; j < f->pbeg[s] + f->pcnt[s]; ++j) {
                    double dx = f->u[3 * i] - f->u[3 * j];
                    double dy = f->u[3 * i + 1] - f->u[3 * j + 1];
                    double dz = f->u[3 * i + 2] - f->u[3 * j + 2];
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 == 0.0) continue;
                    double r = sqrt(r2);
                    ps[i] += qs[j] / r;
                    double w = qs[j] / (r2 * r);
                    gs[3 * i] -= w * dx;
                    gs[3 * i + 1] -= w * dy;
                    gs[3 * i + 2] -= w * dz;
                }
            }
        }
    }

    /* back to caller order and physical units */
    {
        double ih = 1.0 / f->h, ih2 = ih * ih;
        int64_t nout = targets ? nt : N;
        for (int64_t t = 0; t < nout; ++t) {
            int64_t s = targets ? inv[targets[t]] : inv[t];
            phi[t] = ps[s] * ih;
            for (int a = 0; a < 3; ++a) grad[3 * t + a] = gs[3 * s + a] * ih2;
        }
    }
    rc = 0;
done:
    free(qs); free(M); free(L); free(ps); free(gs); free(want); free(need); free(inv);
    free(m2l); free(p2p); free(m2l_off); free(p2p_off);
    return rc;
}

/*
 * Far field of sources with charges cq and (optionally) dipoles cp (3 per
 * source), sorted order: P2M (charge + dipole) on leaves, M2M bottom-up, M2L
 * over the list (targets with need[c] only), L2L top-down.  L is returned
 * zero except on needed cells.
 */
static int orc_far_field(const orc_fmm *f, const double *cq, const double *cp, const char *need,
                         const orc_pair *m2l, const int64_t *m2l_off, double *M, double *L)
{
    const orc_mindex *mi = &f->mi;
    int T = mi->nterms;
    int64_t nc = f->ncells;
    memset(M, 0, (size_t)nc * T * sizeof(double));
    memset(L, 0, (size_t)nc * T * sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < nc; ++c) {
        if (!orc_is_leaf(f, c)) continue;
        double X[3];
        orc_centre_d(f, c, X);
        if (cp)
            orc_p2m_dipole_mi(mi, (int)f->pcnt[c], f->u + 3 * f->pbeg[c], cq + f->pbeg[c],
                              cp + 3 * f->pbeg[c], X, M + c * T);
        else
            orc_p2m_mi(mi, (int)f->pcnt[c], f->u + 3 * f->pbeg[c], cq + f->pbeg[c], X, M + c * T);
    }
    for (int64_t c = nc - 1; c >= 1; --c) {
        double Xc[3], Xp[3];
        int64_t p = f->parent[c];
        orc_centre_d(f, c, Xc);
        orc_centre_d(f, p, Xp);
        orc_m2m_mi(mi, M + c * T, Xc, Xp, M + p * T);
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < nc; ++c) {
        if (!need[c]) continue;
        double Xt[3];
        orc_centre_d(f, c, Xt);
        for (int64_t e = m2l_off[c]; e < m2l_off[c + 1]; ++e) {
            double Xs[3];
            int64_t s = m2l[e].b;
            orc_centre_d(f, s, Xs);
            orc_m2l_mi(mi, M + s * T, Xs, Xt, L + c * T);
        }
    }
    for (int64_t c = 1; c < nc; ++c) {
        if (!need[c]) continue;
        double Xc[3], Xp[3];
        int64_t p = f->parent[c];
        orc_centre_d(f, c, Xc);
        orc_centre_d(f, p, Xp);
        orc_l2l_mi(mi, L + p * T, Xp, Xc, L + c * T);
    }
    return 0;
}

/*
 * FMM adjoint (see the header): for charges q and upstream gradients a = dL/dphi
 * (N, may be NULL) and b = dL/dgrad (N x 3, may be NULL), caller order and
 * physical units, returns dq = dL/dq and dx = dL/dx at all N particles
 * (targets == NULL) or at the nt listed ones.  In normalised coordinates
 * u = (x - c) / h the dipoles are b' = b / h, and then
 *   dq = Psi_u / h,   dx = (a grad_u + H_u b' + q grad Psi_u) / h^2,
 * where Psi_u is the field of charges a and dipoles b' and grad_u, H_u are the
 * gradient and Hessian of the potential of the charges q.  Steps: the far
 * field of q (P2M, M2M, M2L, L2L over the traversal's lists), the far field
 * of (a, b'), then per wanted target L2P of both (gradient, Hessian-vector
 * product, Psi and its gradient) and P2P over the P2P list:
 *   Psi      += a_j / r + b'_j . d / r^3
 *   grad Psi += -a_j d / r^3 + b'_j / r^3 - 3 (b'_j . d) d / r^5
 *   grad     += -q_j d / r^3
 *   H b'_i   += q_j (-b'_i / r^3 + 3 (d . b'_i) d / r^5),      d = u_i - u_j, r != 0.
 */
int orc_backward(orc_fmm *f, const double *q, const double *a, const double *b, int64_t nt,
                 const int64_t *targets, double *dq, double *dx)
{
    if (!f->built) return -1;
    const orc_mindex *mi = &f->mi;
    int T = mi->nterms;
    int64_t N = f->N, nc = f->ncells;
    double ih = 1.0 / f->h, ih2 = ih * ih;
    double *qs = (double *)malloc((size_t)N * sizeof(double));
    double *as = (double *)calloc((size_t)N, sizeof(double));
    double *bs = (double *)calloc((size_t)N * 3, sizeof(double));
    double *Mq = (double *)malloc((size_t)nc * T * sizeof(double));
    double *Lq = (double *)malloc((size_t)nc * T * sizeof(double));
    double *Ma = (double *)malloc((size_t)nc * T * sizeof(double));
    double *La = (double *)malloc((size_t)nc * T * sizeof(double));
    double *out_q = (double *)calloc((size_t)N, sizeof(double));
    double *out_x = (double *)calloc((size_t)N * 3, sizeof(double));
    char *want = (char *)calloc((size_t)N, 1);
    char *need = (char *)calloc((size_t)nc, 1);
    int64_t *inv = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    orc_pair *m2l = NULL, *p2p = NULL;
    int64_t *m2l_off = NULL, *p2p_off = NULL;
    int rc = -1;
    if (!qs || !as || !bs || !Mq || !Lq || !Ma || !La || !out_q || !out_x || !want || !need || !inv)
        goto done;
    for (int64_t s = 0; s < N; ++s) {
        int64_t i = f->perm[s];
        qs[s] = q[i];
        inv[i] = s;
        if (a) as[s] = a[i];
        if (b) for (int c = 0; c < 3; ++c) bs[3 * s + c] = b[3 * i + c] * ih;
    }
    if (targets) {
        for (int64_t t = 0; t < nt; ++t) {
            if (targets[t] < 0 || targets[t] >= N) goto done;
            want[inv[targets[t]]] = 1;
        }
    } else {
        memset(want, 1, (size_t)N);
    }
    for (int64_t c = nc - 1; c >= 0; --c) {
        if (orc_is_leaf(f, c)) {
            for (int64_t j = f->pbeg[c]; j < f->pbeg[c] + f->pcnt[c]; ++j)
                if (want[j]) { need[c] = 1; break; }
        }
        if (need[c] && f->parent[c] >= 0) need[f->parent[c]] = 1;
    }
    m2l = (orc_pair *)malloc((size_t)(f->m2l.n + 1) * sizeof(orc_pair));
    m2l_off = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    p2p = (orc_pair *)malloc((size_t)(f->p2p.n + 1) * sizeof(orc_pair));
    p2p_off = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
    if (!m2l || !m2l_off || !p2p || !p2p_off) goto done;
    memcpy(m2l, f->m2l.v, (size_t)f->m2l.n * sizeof(orc_pair));
    qsort(m2l, (size_t)f->m2l.n, sizeof(orc_pair), orc_cmp_pair);
    for (int64_t e = 0; e < f->m2l.n; ++e) m2l_off[m2l[e].a + 1]++;
    for (int64_t c = 0; c < nc; ++c) m2l_off[c + 1] += m2l_off[c];
    memcpy(p2p, f->p2p.v, (size_t)f->p2p.n * sizeof(orc_pair));
    qsort(p2p, (size_t)f->p2p.n, sizeof(orc_pair), orc_cmp_pair);
    for (int64_t e = 0; e < f->p2p.n; ++e) p2p_off[p2p[e].a + 1]++;
    for (int64_t c = 0; c < nc; ++c) p2p_off[c + 1] += p2p_off[c];

    orc_far_field(f, qs, NULL, need, m2l, m2l_off, Mq, Lq);
    orc_far_field(f, as, bs, need, m2l, m2l_off, Ma, La);

#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t c = 0; c < nc; ++c) {
        if (!orc_is_leaf(f, c) || !need[c]) continue;
        double Xt[3];
        orc_centre_d(f, c, Xt);
        for (int64_t i = f->pbeg[c]; i < f->pbeg[c] + f->pcnt[c]; ++i) {
            if (!want[i]) continue;
            const double *ui = f->u + 3 * i, *bi = bs + 3 * i;
            double phi_q = 0.0, g[3] = {0.0, 0.0, 0.0}, hb[3] = {0.0, 0.0, 0.0};
            double psi = 0.0, gpsi[3] = {0.0, 0.0, 0.0};
            orc_l2p_mi(mi, Lq + c * T, Xt, 1, ui, &phi_q, g);
            orc_l2p_hess_mi(mi, Lq + c * T, Xt, ui, bi, hb);
            orc_l2p_mi(mi, La + c * T, Xt, 1, ui, &psi, gpsi);
            for (int64_t e = p2p_off[c]; e < p2p_off[c + 1]; ++e) {
                int64_t s = p2p[e].b;
                for (int64_t j = f->pbeg[s]; j < f->pbeg[s] + f->pcnt[s]; ++j) {
                    const double *uj = f->u + 3 * j, *bj = bs + 3 * j;
                    double d[3] = {ui[0] - uj[0], ui[1] - uj[1], ui[2] - uj[2]};
                    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    if (r2 == 0.0) continue;
                    double r = sqrt(r2), r3 = r2 * r, r5 = r3 * r2;
                    double bjd = bj[0] * d[0] + bj[1] * d[1] + bj[2] * d[2];
                    double bid = bi[0] * d[0] + bi[1] * d[1] + bi[2] * d[2];
                    psi += as[j] / r + bjd / r3;
                    for (int k = 0; k < 3; ++k) {
                        gpsi[k] += -as[j] * d[k] / r3 + bj[k] / r3 - 3.0 * bjd * d[k] / r5;
                        g[k] += -qs[j] * d[k] / r3;
                        hb[k] += qs[j] * (-bi[k] / r3 + 3.0 * bid * d[k] / r5);
                    }
                }
            }
            out_q[i] = psi * ih;
            for (int k = 0; k < 3; ++k) out_x[3 * i + k] = (as[i] * g[k] + hb[k] + qs[i] * gpsi[k]) * ih2;
        }
    }
    {
        int64_t nout = targets ? nt : N;
        for (int64_t t = 0; t < nout; ++t) {
            int64_t s = targets ? inv[targets[t]] : inv[t];
            dq[t] = out_q[s];
            for (int k = 0; k < 3; ++k) dx[3 * t + k] = out_x[3 * s + k];
        }
    }
    rc = 0;
done:
    free(qs); free(as); free(bs); free(Mq); free(Lq); free(Ma); free(La); free(out_q); free(out_x);
    free(want); free(need); free(inv); free(m2l); free(p2p); free(m2l_off); free(p2p_off);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Introspection for the tests.                                        */
/* ------------------------------------------------------------------ */

/* Canonical cell id, independent of array order: (1 << 3*level) | prefix. */
static uint64_t orc_canon(const orc_fmm *f, int64_t c)
{
    return ((uint64_t)1 << (3 * f->level[c])) | f->prefix[c];
}

int64_t orc_ncells(const orc_fmm *f) { return f->ncells; }
int64_t orc_nm2l(const orc_fmm *f) { return f->m2l.n; }
int64_t orc_np2p(const orc_fmm *f) { return f->p2p.n; }

void orc_norm(const orc_fmm *f, double *centre, double *h)
{
    for (int a = 0; a < 3; ++a) centre[a] = f->centre[a];
    *h = f->h;
}

void orc_sorted(const orc_fmm *f, uint64_t *key, int64_t *perm, double *u, float *u32)
{
    int64_t N = f->N;
    if (key) memcpy(key, f->key, (size_t)N * sizeof(uint64_t));
    if (perm) memcpy(perm, f->perm, (size_t)N * sizeof(int64_t));
    if (u) memcpy(u, f->u, (size_t)N * 3 * sizeof(double));
    if (u32) memcpy(u32, f->u32, (size_t)N * 3 * sizeof(float));
}

void orc_cells(const orc_fmm *f, uint64_t *canon, int32_t *level, int64_t *pbeg, int64_t *pcnt,
               int32_t *nchild, int64_t *parent, float *centre, float *radius)
{
    for (int64_t c = 0; c < f->ncells; ++c) {
        if (canon) canon[c] = orc_canon(f, c);
        if (level) level[c] = f->level[c];
        if (pbeg) pbeg[c] = f->pbeg[c];
        if (pcnt) pcnt[c] = f->pcnt[c];
        if (nchild) nchild[c] = f->ccnt[c];
        if (parent) parent[c] = f->parent[c];
        if (centre) for (int a = 0; a < 3; ++a) centre[3 * c + a] = f->cx[3 * c + a];
        if (radius) radius[c] = f->radius[c];
    }
}

/* Lists as canonical (target, source) id pairs, 2 x n each, in traversal order. */
void orc_lists(const orc_fmm *f, uint64_t *m2l, uint64_t *p2p)
{
    if (m2l)
        for (int64_t e = 0; e < f->m2l.n; ++e) {
            m2l[2 * e] = orc_canon(f, f->m2l.v[e].a);
            m2l[2 * e + 1] = orc_canon(f, f->m2l.v[e].b);
        }
    if (p2p)
        for (int64_t e = 0; e < f->p2p.n; ++e) {
            p2p[2 * e] = orc_canon(f, f->p2p.v[e].a);
            p2p[2 * e + 1] = orc_canon(f, f->p2p.v[e].b);
        }
}

/* Lists as cell-index pairs (indices into orc_cells), 2 x n each. */
void orc_lists_idx(const orc_fmm *f, int64_t *m2l, int64_t *p2p)
{
    if (m2l)
        for (int64_t e = 0; e < f->m2l.n; ++e) {
            m2l[2 * e] = f->m2l.v[e].a;
            m2l[2 * e + 1] = f->m2l.v[e].b;
        }
    if (p2p)
        for (int64_t e = 0; e < f->p2p.n; ++e) {
            p2p[2 * e] = f->p2p.v[e].a;
            p2p[2 * e + 1] = f->p2p.v[e].b;
        }
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
