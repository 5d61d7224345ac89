"""The seeded input recipe: each generator draws the distribution it states.

The workloads are synthetic stand-ins for the paper's particle sets (random
points in a cube, Sec. 3.4; a Plummer sphere for adaptive trees; Gaussian
charge vectors; lognormal system sizes), so these checks pin the sampling
against closed forms: ranges, moments, the Plummer cumulative mass profile
M(<r) = r^3 / (1 + r^2)^(3/2) truncated at r = 100, isotropy, and the
lognormal size law.  Everything runs on the CPU.
"""
import numpy as np
import pytest

from paper_1209_3516_gb300 import inputs


def test_uniform_cube_ranges_and_moments():
    x, q = inputs.uniform_cube(200000)
    assert x.shape == (200000, 3) and q.shape == (200000,)
    assert x.dtype == np.float64 and q.dtype == np.float64
    assert x.min() >= 0.0 and x.max() < 1.0
    assert q.min() >= -1.0 and q.max() < 1.0
    # U[0,1): mean 1/2, variance 1/12; U[-1,1): mean 0, variance 1/3 (5 sigma bands)
    n = x.shape[0]
    assert np.all(np.abs(x.mean(axis=0) - 0.5) < 5 * np.sqrt(1 / 12 / n))
    assert np.all(np.abs(x.var(axis=0) - 1 / 12) < 0.01)
    assert abs(q.mean()) < 5 * np.sqrt(1 / 3 / n)
    assert abs(q.var() - 1 / 3) < 0.01


def test_generators_are_seeded():
    a, qa = inputs.uniform_cube(1000, 7)
    b, qb = inputs.uniform_cube(1000, 7)
    c, _ = inputs.uniform_cube(1000, 8)
    assert np.array_equal(a, b) and np.array_equal(qa, qb)
    assert not np.array_equal(a, c)
    assert np.array_equal(inputs.plummer(500)[0], inputs.plummer(500)[0])
    assert np.array_equal(inputs.lognormal_sizes(64), inputs.lognormal_sizes(64))


def test_plummer_mass_profile_and_isotropy():
    from scipy import stats

    N, rmax = 200000, 100.0
    x, q = inputs.plummer(N)
    assert x.shape == (N, 3) and np.all(q == 1.0 / N)
    r = np.linalg.norm(x, axis=1)
    assert r.max() <= rmax

    def cdf(s):
        m = lambda t: t ** 3 / (1.0 + t * t) ** 1.5
        return m(np.asarray(s)) / m(rmax)

    res = stats.kstest(r, cdf)
    assert res.pvalue > 1e-3, res
    # half-mass radius of the untruncated sphere: (2^(2/3) - 1)^(-1/2) = 1.305
    assert abs(np.median(r) - 1.0 / np.sqrt(2 ** (2 / 3) - 1)) < 0.02
    u = x / r[:, None]
    assert np.all(np.abs(u.mean(axis=0)) < 5 / np.sqrt(3 * N))   # isotropic: E[u] = 0, Var = 1/3
    assert stats.kstest(u[:, 2], stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-3   # cos(theta) uniform


def test_gaussian_charge_vectors():
    g = inputs.gaussian_charges(100000, 4)
    assert g.shape == (4, 100000)
    assert np.all(np.abs(g.mean(axis=1)) < 5 / np.sqrt(100000))
    assert np.all(np.abs(g.std(axis=1) - 1.0) < 0.01)


@pytest.mark.parametrize("nsys", [64, 20000])
def test_lognormal_system_sizes(nsys):
    lo, hi = 1000, 200000
    n = inputs.lognormal_sizes(nsys, lo, hi)
    assert n.dtype == np.int64 and n.shape == (nsys,)
    assert n.min() >= lo and n.max() <= hi
    if nsys >= 10000:
        # geometric-mean centre sqrt(lo hi); +-2 sigma spans [lo, hi], so ~2.3 % clamp at each end
        logn = np.log(n)
        assert abs(np.median(logn) - 0.5 * np.log(lo * hi)) < 0.05
        s = 0.25 * np.log(hi / lo)
        inner = logn[(n > lo) & (n < hi)]
        assert abs(np.mean(n == lo) - 0.02275) < 0.006 and abs(np.mean(n == hi) - 0.02275) < 0.006
        assert abs(np.std(inner) - s * 0.880) < 0.05 * s   # sd of a normal truncated at +-2 sigma


def test_error_sample_is_every_256th_target_at_1m():
    t = inputs.sample_targets(1 << 20)
    assert t.size == 4096 and t[0] == 0 and np.all(np.diff(t) == 256)
    assert inputs.sample_targets(1000).size == 1000
