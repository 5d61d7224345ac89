"""Pins of the oracle's direct sum (the plain definition the FMM approximates).

Kernel (Sec. 3.2, Table 3 caption): phi_i = sum_j q_j / r_ij and
grad_i = -sum_j q_j (x_i - x_j) / r_ij^3.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1209_3516_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _frac(s):
    return float(Fraction(s))


def test_two_particles_closed_form():
    x = np.array([[0.1, -0.2, 0.3], [1.1, 0.4, -0.9]])
    q = np.array([0.7, -1.3])
    phi, g = oracle.direct(x, q)
    d = x[0] - x[1]
    r = np.sqrt(d @ d)
    assert phi[0] == pytest.approx(q[1] / r, rel=1e-15)
    assert phi[1] == pytest.approx(q[0] / r, rel=1e-15)
    np.testing.assert_allclose(g[0], -q[1] * d / r**3, rtol=1e-14)
    np.testing.assert_allclose(g[1], q[0] * d / r**3, rtol=1e-14)


def test_three_particles_hand_worked():
    rows = []
    with open(os.path.join(GOLDEN, "direct_n3.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            a, b, c = line.split("|")
            rows.append(([float(v) for v in a.split()], _frac(b.strip()),
                         [_frac(v) for v in c.split()]))
    x = np.array([r[0][:3] for r in rows])
    q = np.array([r[0][3] for r in rows])
    phi, g = oracle.direct(x, q)
    np.testing.assert_allclose(phi, [r[1] for r in rows], rtol=1e-15, atol=1e-16)
    np.testing.assert_allclose(g, [r[2] for r in rows], rtol=1e-14, atol=1e-16)


def test_coincident_points_contribute_nothing():
    x = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.5], [1.5, 0.5, 0.5]])
    q = np.array([1.0, 2.0, 4.0])
    phi, g = oracle.direct(x, q)
    assert phi[0] == pytest.approx(4.0)
    assert phi[1] == pytest.approx(4.0)
    assert phi[2] == pytest.approx(3.0)
    np.testing.assert_allclose(g[0], [4.0, 0, 0])
    np.testing.assert_allclose(g[2], [-3.0, 0, 0])


def test_force_balance_and_homogeneity():
    x, q = inputs.uniform_cube(700, 11)
    phi, g = oracle.direct(x, q)
    # Newton's third law: sum_i q_i grad_i = 0 for the exact field
    bal = (q[:, None] * g).sum(0)
    scale = np.abs(q[:, None] * g).sum()
    assert np.abs(bal).max() < 1e-13 * scale
    # homogeneity of degree -1: x -> 2x + shift gives phi/2, grad/4
    phi2, g2 = oracle.direct(2.0 * x + 3.25, q)
    np.testing.assert_allclose(phi2, phi / 2, rtol=1e-12)
    np.testing.assert_allclose(g2, g / 4, rtol=1e-11, atol=1e-12 * np.abs(g).max())


def test_target_subset_matches_full():
    x, q = inputs.uniform_cube(900, 12)
    phi, g = oracle.direct(x, q)
    t = np.array([0, 5, 899, 450, 5])
    ps, gs = oracle.direct(x, q, t)
    np.testing.assert_array_equal(ps, phi[t])
    np.testing.assert_array_equal(gs, g[t])


def test_brute_force_python():
    x, q = inputs.uniform_cube(60, 13)
    phi, g = oracle.direct(x, q)
    for i in (0, 17, 59):
        p = 0.0
        gg = np.zeros(3)
        for j in range(60):
            if j == i:
                continue
            d = x[i] - x[j]
            r = float(np.sqrt(d @ d))
            p += q[j] / r
            gg -= q[j] * d / r**3
        assert phi[i] == pytest.approx(p, rel=1e-13)
        np.testing.assert_allclose(g[i], gg, rtol=1e-12)
