"""Pins of the oracle's adjoint (derivatives of the Laplace sums).

dL/dq and dL/dx for L = sum_i a_i phi_i + sum_i b_i . grad_i are pinned by
FP64 central finite differences of the direct sum, a two-particle closed
form and translation invariance (direct adjoint); the dipole P2M and the
Hessian L2P by finite differences of the already pinned charge P2M and
gradient L2P; the FMM adjoint by exact reproduction of the direct adjoint
when every pair is P2P (theta = 0) and by convergence in P.
"""
import numpy as np
import pytest

import oracle
from paper_1209_3516_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


def upstream(N, seed):
    g = inputs.rng(seed)
    return g.standard_normal(N), g.standard_normal((N, 3))


def test_direct_backward_two_particles_closed_form():
    # x_0 = 0, x_1 = (r, 0, 0): phi_0 = q_1 / r, grad_0 = (q_1 / r^2, 0, 0),
    # phi_1 = q_0 / r, grad_1 = (-q_0 / r^2, 0, 0)
    r = 0.7
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    q = np.array([0.3, -1.1])
    a = np.array([0.5, 2.0])
    b = np.array([[0.2, -0.4, 0.9], [1.5, 0.3, -0.7]])
    dq, dx = oracle.direct_backward(x, q, a, b)
    # L = a0 q1 / r + a1 q0 / r + b0x q1 / r^2 - b1x q0 / r^2
    assert np.allclose(dq, [a[1] / r - b[1, 0] / r**2, a[0] / r + b[0, 0] / r**2], rtol=1e-14)
    # along the axis: d/dr of the four terms; dL/dx_0 = -dL/dx_1 (translation)
    dLdr = -(a[0] * q[1] + a[1] * q[0]) / r**2 - 2 * (b[0, 0] * q[1] - b[1, 0] * q[0]) / r**3
    assert np.isclose(dx[1, 0], dLdr, rtol=1e-13)
    assert np.isclose(dx[0, 0], -dLdr, rtol=1e-13)
    # grad_0y = -q_1 (0 - y_1) / r^3 = q_1 y_1 / r^3, grad_1y = -q_0 (y_1 - 0) / r^3
    assert np.isclose(dx[1, 1], (b[0, 1] * q[1] - b[1, 1] * q[0]) / r**3, rtol=1e-13)
    assert np.isclose(dx[1, 2], (b[0, 2] * q[1] - b[1, 2] * q[0]) / r**3, rtol=1e-13)
    assert np.allclose(dx[0], -dx[1], rtol=1e-13)


@pytest.mark.parametrize("N", [200, 8192])
def test_direct_backward_matches_central_differences(N):
    # FP64 central differences, h = 1e-6, of L(x, q) = a . phi + b : grad
    x, q = inputs.uniform_cube(N, 2100 + N)
    a, b = upstream(N, 2200 + N)
    ks = [0, N // 3, N - 1]
    dq, dx = oracle.direct_backward(x, q, a, b, targets=ks)

    def loss(xx, qq):
        p, g = oracle.direct(xx, qq)
        return float(a @ p + np.sum(b * g))

    h = 1e-6
    for t, k in enumerate(ks):
        e = np.zeros(N)
        e[k] = h
        fd = (loss(x, q + e) - loss(x, q - e)) / (2 * h)
        assert abs(fd - dq[t]) <= 1e-6 * abs(dq[t]) + 1e-6, (k, fd, dq[t])
        for c in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, c] += h
            xm[k, c] -= h
            fd = (loss(xp, q) - loss(xm, q)) / (2 * h)
            scale = np.linalg.norm(dx[t])
            assert abs(fd - dx[t, c]) <= 1e-6 * scale, (k, c, fd, dx[t, c])


def test_direct_backward_translation_invariance_and_energy():
    N = 500
    x, q = inputs.uniform_cube(N, 2300)
    a, b = upstream(N, 2301)
    dq, dx = oracle.direct_backward(x, q, a, b)
    # L does not change when every particle moves by the same vector
    assert np.all(np.abs(dx.sum(axis=0)) <= 1e-11 * np.abs(dx).sum(axis=0))
    # L = sum_i q_i phi_i (a = q through phi only): dL/dq = phi, dL/dx = 2 q grad
    phi, g = oracle.direct(x, q)
    dq2, dx2 = oracle.direct_backward(x, q, q, None)
    assert rel(dq2, phi) <= 1e-13
    assert rel(dx2, 2 * q[:, None] * g) <= 1e-13


def test_dipole_p2m_is_the_derivative_of_charge_p2m():
    # a dipole p at y has the multipole sum_c p_c d/dy_c of a unit charge's multipole
    P = 6
    rng = inputs.rng(2400)
    X = np.array([0.1, -0.2, 0.05])
    y = X + rng.random((3, 3)) * 0.3 - 0.15
    a = rng.standard_normal(3)
    p = rng.standard_normal((3, 3))
    M = oracle.p2m_dipole(P, y, a, p, X)
    ref = oracle.p2m(P, y, a, X)
    eps = 1e-5
    for j in range(3):
        for c in range(3):
            yp, ym = y[j].copy(), y[j].copy()
            yp[c] += eps
            ym[c] -= eps
            ref += p[j, c] * (oracle.p2m(P, yp[None], [1.0], X) - oracle.p2m(P, ym[None], [1.0], X)) / (2 * eps)
    assert np.allclose(M, ref, rtol=1e-8, atol=1e-10)
    # degree 0 carries only the charges, degree 1 gets the dipoles: M_{e_c} = sum a d_c + p_c
    assert np.isclose(M[0], a.sum(), rtol=1e-14)


def test_dipole_far_field_converges_to_dipole_potential():
    # P2M(dipole) -> M2L -> L2P approaches p . (x - y) / |x - y|^3 as P grows
    Xs, Xt = np.zeros(3), np.array([1.0, 0.4, -0.3])
    y = np.array([[0.08, -0.05, 0.1]])
    p = np.array([[0.3, -0.7, 0.5]])
    x = Xt + np.array([[-0.06, 0.09, 0.04]])
    d = x[0] - y[0]
    exact = p[0] @ d / np.linalg.norm(d) ** 3
    errs = []
    for P in (3, 5, 7, 9):
        L = oracle.m2l(P, oracle.p2m_dipole(P, y, [0.0], p, Xs), Xs, Xt)
        phi, _ = oracle.l2p(P, L, Xt, x)
        errs.append(abs(phi[0] - exact) / abs(exact))
    assert all(e1 < e0 for e0, e1 in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-5


def test_hessian_l2p_is_the_derivative_of_gradient_l2p():
    P = 6
    rng = inputs.rng(2500)
    L = rng.standard_normal(oracle.nterms(P))
    Xt = np.array([0.3, 0.1, -0.2])
    x = Xt + rng.random(3) * 0.2 - 0.1
    v = rng.standard_normal(3)
    hv = oracle.l2p_hess(P, L, Xt, x, v)
    eps = 1e-6
    _, gp = oracle.l2p(P, L, Xt, (x + eps * v)[None])
    _, gm = oracle.l2p(P, L, Xt, (x - eps * v)[None])
    # the Hessian is symmetric, so H v is the directional derivative of the gradient along v
    assert np.allclose(hv, (gp[0] - gm[0]) / (2 * eps), rtol=1e-7, atol=1e-8)


def test_fmm_backward_theta_zero_is_the_direct_adjoint():
    N = 3000
    x, q = inputs.uniform_cube(N, 2600)
    a, b = upstream(N, 2601)
    f = oracle.FMM(N, 4, 0.0, 32).build(x)
    dq, dx = f.backward(q, a, b)
    rq, rx = oracle.direct_backward(x, q, a, b)
    assert rel(dq, rq) <= 1e-12 and rel(dx, rx) <= 1e-12


def test_fmm_backward_converges_in_p_and_subset_matches():
    N = 6000
    x, q = inputs.uniform_cube(N, 2700)
    a, b = upstream(N, 2701)
    rq, rx = oracle.direct_backward(x, q, a, b)
    eq = []
    for P in (3, 5, 8):
        f = oracle.FMM(N, P, 0.4, 32).build(x)
        dq, dx = f.backward(q, a, b)
        eq.append((rel(dq, rq), rel(dx, rx)))
    assert eq[0][0] > eq[1][0] > eq[2][0], eq
    assert eq[0][1] > eq[2][1], eq
    assert eq[2][0] < 1e-5 and eq[2][1] < 1e-6, eq
    t = inputs.sample_targets(N, 500)
    sq, sx = f.backward(q, a, b, targets=t)
    assert np.array_equal(sq, dq[t]) and np.array_equal(sx, dx[t])


def test_fmm_backward_without_dipoles_reproduces_the_forward_fields():
    # a = q, b = 0: dL/dq is the FMM potential and dL/dx = 2 q grad (the kernel is
    # symmetric), step for step the same operations as the forward evaluation
    N = 4000
    x, q = inputs.uniform_cube(N, 2800)
    f = oracle.FMM(N, 5, 0.45, 24).build(x)
    phi, g = f.evaluate(q)
    dq, dx = f.backward(q, q, None)
    assert rel(dq, phi) <= 1e-15
    assert rel(dx, 2 * q[:, None] * g) <= 1e-15
