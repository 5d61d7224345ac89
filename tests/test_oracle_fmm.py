"""Pins of the oracle FMM as a whole (Sec. 3.1-3.3).

  * theta = 0 accepts no pair, every interaction is P2P: the FMM must equal
    the direct sum up to summation order (Sec. 3.2: shrinking theta turns the
    method into direct summation);
  * the error falls with the order P at fixed theta and with theta at fixed
    P (error O(theta^p), Sec. 3.2);
  * Newton's third law: sum_i q_i grad_i = 0, exactly at theta = 0;
  * Table 3 as a soft anchor: at the paper's (p, theta) pairs the force error
    is of the order the paper prints, and nearly the same along each row;
  * evaluating a subset of targets gives the same numbers as a full run.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1209_3516_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("N,ncrit,P,kind", [(1, 64, 4, "u"), (2, 64, 4, "u"), (64, 64, 4, "u"),
                                            (65, 64, 3, "u"), (3000, 16, 6, "u"),
                                            (2500, 8, 4, "p")])
def test_theta_zero_reproduces_direct_sum(N, ncrit, P, kind):
    x, q = inputs.uniform_cube(N, 51) if kind == "u" else inputs.plummer(N, 52)
    if kind == "p":
        q = inputs.rng(53).random(N) - 0.5
    pd, gd = oracle.direct(x, q)
    f = oracle.FMM(N, P, 0.0, ncrit).build(x)
    p, g = f.evaluate(q)
    if N == 1:
        assert p[0] == 0.0 and np.all(g == 0.0)
        return
    assert rel_l2(p, pd) < 1e-13
    assert rel_l2(g, gd) < 1e-13


def test_error_falls_with_order():
    N = 6000
    x, q = inputs.uniform_cube(N, 54)
    pd, gd = oracle.direct(x, q)
    errs = []
    for P in (2, 3, 4, 5, 6, 8, 10):
        p, g = oracle.FMM(N, P, 0.4, 32).build(x).evaluate(q)
        errs.append((rel_l2(p, pd), rel_l2(g, gd)))
    errs = np.array(errs)
    assert np.all(np.diff(errs[:, 0]) < 0)
    assert np.all(np.diff(errs[:, 1]) < 0)
    assert errs[-1, 1] < 1e-3 * errs[0, 1]


def test_error_falls_with_theta():
    N = 6000
    x, q = inputs.uniform_cube(N, 55)
    pd, gd = oracle.direct(x, q)
    errs = []
    for th in (0.8, 0.6, 0.5, 0.4, 0.3, 0.2):
        p, g = oracle.FMM(N, 4, th, 32).build(x).evaluate(q)
        errs.append((rel_l2(p, pd), rel_l2(g, gd)))
    errs = np.array(errs)
    assert np.all(np.diff(errs[:, 1]) < 0)
    assert np.all(np.diff(errs[:, 0]) < 0)
    # O(theta^p)-like: halving theta from 0.4 to 0.2 gains well over a factor 2^2
    assert errs[3, 1] / errs[5, 1] > 4.0


def test_force_balance():
    N = 4000
    x, q = inputs.uniform_cube(N, 56)
    scale = None
    for th, tol in ((0.0, 1e-13), (0.4, 1e-4)):
        p, g = oracle.FMM(N, 6, th, 32).build(x).evaluate(q)
        bal = np.abs((q[:, None] * g).sum(0)).max()
        scale = np.abs(q[:, None] * g).sum()
        assert bal < tol * scale, (th, bal / scale)


def test_subset_equals_full_run():
    N = 5000
    x, q = inputs.uniform_cube(N, 57)
    f = oracle.FMM(N, 4, 0.45, 24).build(x)
    p, g = f.evaluate(q)
    t = inputs.sample_targets(N, 300)
    ps, gs = f.evaluate(q, t)
    np.testing.assert_array_equal(ps, p[t])
    np.testing.assert_array_equal(gs, g[t])


def test_input_order_and_frame_invariance():
    N = 3000
    x, q = inputs.uniform_cube(N, 58)
    p, g = oracle.FMM(N, 4, 0.4, 32).build(x).evaluate(q)
    perm = inputs.rng(59).permutation(N)
    p2, g2 = oracle.FMM(N, 4, 0.4, 32).build(x[perm]).evaluate(q[perm])
    np.testing.assert_allclose(p2, p[perm], rtol=1e-12, atol=1e-12 * np.abs(p).max())
    np.testing.assert_allclose(g2, g[perm], rtol=1e-11, atol=1e-12 * np.abs(g).max())
    # scaling by a power of two and shifting: the normalised problem is the same
    p3, g3 = oracle.FMM(N, 4, 0.4, 32).build(4.0 * x - 7.0).evaluate(q)
    np.testing.assert_allclose(p3, p / 4.0, rtol=1e-11, atol=1e-12 * np.abs(p).max())
    np.testing.assert_allclose(g3, g / 16.0, rtol=1e-10, atol=1e-12 * np.abs(g).max())


def test_energy_is_half_charge_potential_sum():
    N = 2000
    x, q = inputs.uniform_cube(N, 60)
    pd, _ = oracle.direct(x, q)
    p, _ = oracle.FMM(N, 8, 0.3, 32).build(x).evaluate(q)
    E = 0.5 * float(q @ p)
    Ed = 0.5 * float(q @ pd)
    # pairwise energy from its own definition: sum over i < j of q_i q_j / r_ij
    d = x[:, None, :] - x[None, :, :]
    r = np.sqrt((d * d).sum(-1))
    iu = np.triu_indices(N, 1)
    Epair = float((q[:, None] * q[None, :])[iu] @ (1.0 / r[iu]))
    assert Ed == pytest.approx(Epair, rel=1e-11)
    assert E == pytest.approx(Epair, rel=1e-5)


def _table3():
    rows = []
    with open(os.path.join(GOLDEN, "table3_ptheta.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            e, p, th, t = line.split()
            rows.append((float(e), int(p), float(th), float(t)))
    return rows


@pytest.mark.slow
def test_table3_soft_anchor():
    # N = 1e5, N_crit = 30 as in Table 3; error measured on a 4,000-target sample.
    # The paper does not define its MAC radius, expansion centre or charges
    # exactly, so only the structure is pinned: along each row of Table 3 the
    # error is nearly constant, successive rows differ by about the printed
    # factor of 10, and the level is the printed one within a loose band
    # (this reading lands 3-10x above the printed Err).
    N = 100000
    x, q = inputs.uniform_cube(N, 61)
    t = inputs.sample_targets(N, 4000)
    pd, gd = oracle.direct(x, q, t)
    by_row = {}
    for err, P, th, _ in _table3():
        if err < 1e-4:
            continue  # the 1e-5 row needs theta as small as 0.12: too slow for the CPU suite
        _, g = oracle.FMM(N, P, th, 30).build(x).evaluate(q, t)
        e = rel_l2(g, gd)
        by_row.setdefault(err, []).append(e)
        assert err / 5 < e < err * 20, (err, P, th, e)
    for err, es in by_row.items():
        es = np.array(es)
        assert es.max() / es.min() < 2.5, (err, es)
    ratio = np.mean(by_row[1e-3]) / np.mean(by_row[1e-4])
    assert 4.0 < ratio < 25.0, ratio


def test_hybrid_accuracy_stays_within_the_mac_bound():
    # moving MAC-passing leaf pairs from P2P to M2L keeps the error of the same
    # order (the MAC bounds every M2L pair) and it still falls with P
    N = 20000
    x, q = inputs.uniform_cube(N, 2900)
    pd, gd = oracle.direct(x, q)
    errs = {}
    for P in (4, 6, 8):
        for hyb in (-1, 0):
            pr, gr = oracle.FMM(N, P, 0.5, 32, hybrid_min_pairs=hyb).build(x).evaluate(q)
            errs[(P, hyb)] = (np.linalg.norm(pr - pd) / np.linalg.norm(pd), np.linalg.norm(gr - gd) / np.linalg.norm(gd))
    for P in (4, 6, 8):
        assert errs[(P, 0)][0] <= 5 * errs[(P, -1)][0] and errs[(P, 0)][1] <= 5 * errs[(P, -1)][1], errs
    assert errs[(4, 0)][1] > errs[(6, 0)][1] > errs[(8, 0)][1]
    pr0, gr0 = oracle.FMM(N, 4, 0.0, 32, hybrid_min_pairs=0).build(x).evaluate(q)
    assert np.linalg.norm(pr0 - pd) / np.linalg.norm(pd) < 1e-13   # theta = 0: the MAC never passes
