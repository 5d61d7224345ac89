"""Pins of the oracle's Cartesian Taylor expansions (Sec. 3.1, Table 1).

Each operator is checked against something other than its own formula:
exact symbolic derivatives, closed forms, re-expansion identities that hold
exactly for the truncated series, finite differences, and convergence to the
direct interaction at the rate ((B_A + B_B) / R)^p of Sec. 3.2.
"""
import numpy as np
import pytest

import oracle

rng = np.random.default_rng(20120916)


def _index(P):
    k = oracle.multi_indices(P)
    return {tuple(int(v) for v in row): i for i, row in enumerate(k)}, k


def test_multi_index_count_and_uniqueness():
    for P in range(1, 11):
        idx, k = _index(P)
        assert len(k) == P * (P + 1) * (P + 2) // 6
        assert len(idx) == len(k)
        assert k.sum(1).max() == P - 1


def test_taylor_closed_forms():
    R = np.array([0.3, -0.7, 1.1])
    r = np.linalg.norm(R)
    idx, _ = _index(3)
    b = oracle.taylor(3, R)
    assert b[idx[(0, 0, 0)]] == pytest.approx(1 / r, rel=1e-15)
    for a, e in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
        assert b[idx[e]] == pytest.approx(-R[a] / r**3, rel=1e-14)
    # second derivatives / 2!:  (3 R_a^2 / r^5 - 1/r^3) / 2  and  3 R_a R_b / r^5
    assert b[idx[(2, 0, 0)]] == pytest.approx((3 * R[0] ** 2 / r**5 - 1 / r**3) / 2, rel=1e-13)
    assert b[idx[(0, 0, 2)]] == pytest.approx((3 * R[2] ** 2 / r**5 - 1 / r**3) / 2, rel=1e-13)
    assert b[idx[(1, 1, 0)]] == pytest.approx(3 * R[0] * R[1] / r**5, rel=1e-13)
    assert b[idx[(0, 1, 1)]] == pytest.approx(3 * R[1] * R[2] / r**5, rel=1e-13)


def test_taylor_against_symbolic_derivatives():
    sp = pytest.importorskip("sympy")
    P = 8
    X, Y, Z = sp.symbols("X Y Z", real=True)
    f = 1 / sp.sqrt(X**2 + Y**2 + Z**2)
    point = {X: sp.Rational(3, 7), Y: sp.Rational(-2, 5), Z: sp.Rational(5, 6)}
    R = np.array([3 / 7, -2 / 5, 5 / 6])
    idx, k = _index(P)
    b = oracle.taylor(P, R)
    derivs = {(0, 0, 0): f}
    for t in range(len(k)):
        m = tuple(int(v) for v in k[t])
        if m not in derivs:
            a = next(i for i in range(3) if m[i] > 0)
            lower = list(m)
            lower[a] -= 1
            derivs[m] = sp.diff(derivs[tuple(lower)], (X, Y, Z)[a])
        fact = sp.factorial(m[0]) * sp.factorial(m[1]) * sp.factorial(m[2])
        exact = float(sp.N(derivs[m].subs(point) / fact, 30))
        assert b[t] == pytest.approx(exact, rel=2e-13, abs=1e-13 * abs(b[0])), m


def test_taylor_harmonic_and_homogeneous():
    # Laplace: sum_d (m_d+1)(m_d+2) b_{m+2e_d} = 0 ; homogeneity: b_m(2R) = 2^-(|m|+1) b_m(R)
    P = 9
    idx, k = _index(P)
    R = np.array([-0.45, 0.2, 0.9])
    b = oracle.taylor(P, R)
    b2 = oracle.taylor(P, 2 * R)
    for t, m in enumerate(k):
        m = tuple(int(v) for v in m)
        assert b2[t] == pytest.approx(b[t] * 2.0 ** (-(sum(m) + 1)), rel=1e-13, abs=1e-300)
        if sum(m) + 2 <= P - 1:
            s = 0.0
            scale = 0.0
            for d in range(3):
                mm = list(m)
                mm[d] += 2
                term = (m[d] + 1) * (m[d] + 2) * b[idx[tuple(mm)]]
                s += term
                scale += abs(term)
            assert abs(s) <= 1e-12 * scale


def test_p2m_low_moments():
    P = 3
    idx, _ = _index(P)
    y = rng.uniform(-0.2, 0.2, (9, 3)) + np.array([0.5, 0.5, 0.5])
    q = rng.uniform(-1, 1, 9)
    X = np.array([0.55, 0.45, 0.5])
    M = oracle.p2m(P, y, q, X)
    d = y - X
    assert M[idx[(0, 0, 0)]] == pytest.approx(q.sum(), rel=1e-14)
    assert M[idx[(1, 0, 0)]] == pytest.approx((q * d[:, 0]).sum(), rel=1e-13)
    assert M[idx[(0, 0, 2)]] == pytest.approx((q * d[:, 2] ** 2).sum() / 2, rel=1e-13)
    assert M[idx[(1, 1, 0)]] == pytest.approx((q * d[:, 0] * d[:, 1]).sum(), rel=1e-13)


@pytest.mark.parametrize("P", [2, 4, 6, 9])
def test_m2m_is_exact_reexpansion(P):
    # shifting a truncated multipole loses nothing: M2M(P2M about X_C) == P2M about X_P
    y = rng.uniform(-0.1, 0.1, (13, 3)) + np.array([0.3, -0.2, 0.1])
    q = rng.uniform(-1, 1, 13)
    Xc = np.array([0.31, -0.21, 0.12])
    Xp = np.array([0.25, -0.15, 0.05])
    Mc = oracle.p2m(P, y, q, Xc)
    Mp = oracle.m2m(P, Mc, Xc, Xp)
    ref = oracle.p2m(P, y, q, Xp)
    np.testing.assert_allclose(Mp, ref, rtol=1e-12, atol=1e-15 * np.abs(ref).max())


@pytest.mark.parametrize("P", [2, 4, 6, 9])
def test_l2l_is_exact_reexpansion(P):
    # a local expansion is a polynomial of degree P-1; L2L re-centres it exactly
    T = P * (P + 1) * (P + 2) // 6
    Lp = rng.standard_normal(T)
    Xp = np.array([0.1, 0.2, -0.3])
    Xc = np.array([0.15, 0.12, -0.27])
    Lc = oracle.l2l(P, Lp, Xp, Xc)
    pts = Xc + rng.uniform(-0.05, 0.05, (7, 3))
    p1, g1 = oracle.l2p(P, Lp, Xp, pts)
    p2, g2 = oracle.l2p(P, Lc, Xc, pts)
    np.testing.assert_allclose(p2, p1, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(g2, g1, rtol=1e-11, atol=1e-12)


def test_l2p_gradient_is_derivative_of_potential():
    P = 6
    T = P * (P + 1) * (P + 2) // 6
    L = rng.standard_normal(T)
    Xt = np.array([0.0, 0.1, 0.2])
    pts = Xt + rng.uniform(-0.3, 0.3, (5, 3))
    _, g = oracle.l2p(P, L, Xt, pts)
    h = 1e-6
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        pp, _ = oracle.l2p(P, L, Xt, pts + e)
        pm, _ = oracle.l2p(P, L, Xt, pts - e)
        np.testing.assert_allclose(g[:, a], (pp - pm) / (2 * h), rtol=1e-6, atol=1e-8)


def _cluster_pair(rho):
    """Source and target clusters of radius a, centres R apart, (a+a)/R = rho."""
    a = 0.1
    R = 2 * a / rho
    Xs = np.array([0.0, 0.0, 0.0])
    direction = np.array([0.48, -0.6, 0.64])
    Xt = Xs + R * direction / np.linalg.norm(direction)
    y = Xs + rng.uniform(-1, 1, (40, 3)) * a / np.sqrt(3)
    x = Xt + rng.uniform(-1, 1, (25, 3)) * a / np.sqrt(3)
    q = rng.uniform(-1, 1, 40)
    return Xs, Xt, y, q, x


def _exact(y, q, x):
    d = x[:, None, :] - y[None, :, :]
    r = np.sqrt((d * d).sum(-1))
    phi = (q[None, :] / r).sum(1)
    grad = -(q[None, :, None] * d / r[..., None] ** 3).sum(1)
    return phi, grad


@pytest.mark.parametrize("rho", [0.25, 0.5])
def test_m2l_converges_at_the_mac_rate(rho):
    Xs, Xt, y, q, x = _cluster_pair(rho)
    pe, ge = _exact(y, q, x)
    errs = []
    for P in range(1, 12):
        M = oracle.p2m(P, y, q, Xs)
        L = oracle.m2l(P, M, Xs, Xt)
        p, g = oracle.l2p(P, L, Xt, x)
        errs.append((np.linalg.norm(p - pe) / np.linalg.norm(pe),
                     np.linalg.norm(g - ge) / np.linalg.norm(ge)))
    errs = np.array(errs)
    # error of order rho^P (Sec. 3.2): bounded by C rho^P and shrinking by ~rho per order
    for P in range(1, 12):
        assert errs[P - 1, 0] <= 3.0 * rho ** P, (P, errs[P - 1])
        assert errs[P - 1, 1] <= 6.0 * rho ** (P - 1), (P, errs[P - 1])
    assert errs[-1, 0] < 1e-3 * errs[2, 0]
    ratio = np.exp(np.polyfit(np.arange(3, 11), np.log(errs[2:10, 0]), 1)[0])
    assert ratio < 0.9 * rho ** 0.5


def test_single_particle_m2l_limit():
    # one source, one target: P2M -> M2L -> L2P tends to q / |x - y|
    y = np.array([[0.03, -0.02, 0.01]])
    q = np.array([1.7])
    x = np.array([[1.02, 0.97, -0.03]])
    Xs = np.zeros(3)
    Xt = np.array([1.0, 1.0, 0.0])
    exact = q[0] / np.linalg.norm(x[0] - y[0])
    prev = np.inf
    for P in range(1, 10):
        L = oracle.m2l(P, oracle.p2m(P, y, q, Xs), Xs, Xt)
        p, _ = oracle.l2p(P, L, Xt, x)
        err = abs(p[0] - exact) / exact
        assert err < prev or err < 1e-15
        prev = err
    assert prev < 1e-12


def test_m2l_sign_of_a_dipole():
    # +q at +d, -q at -d along x: far field on the +x axis is 2 q d / r^2 > 0
    d = 0.01
    y = np.array([[d, 0, 0], [-d, 0, 0]])
    q = np.array([1.0, -1.0])
    Xs = np.zeros(3)
    Xt = np.array([2.0, 0, 0])
    L = oracle.m2l(3, oracle.p2m(3, y, q, Xs), Xs, Xt)
    p, g = oracle.l2p(3, L, Xt, Xt[None, :])
    assert p[0] == pytest.approx(2 * d / 4.0, rel=1e-3)
    assert g[0, 0] == pytest.approx(-4 * d / 8.0, rel=1e-3)
