"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method: it only draws particle sets.
Both the GPU path (through the tests and the benchmark) and the CPU oracle
receive the arrays it returns; neither generates its own.

Workloads (all FP64 positions, seeds 1209 + workload id, NumPy Philox):
  * uniform cube: x ~ U[0,1)^3, q ~ U[-1,1)   ("randomly distributed particles
    in a cube", Sec. 3.4 and the caption of Fig. 3);
  * Plummer sphere, scale radius 1, truncated at r = 100, equal charges 1/N
    (radius by inverse-CDF sampling r = (X^(-2/3) - 1)^(-1/2), X ~ U(0,1),
    isotropic direction);
  * Gaussian charge vectors q ~ N(0,1) for the many-right-hand-side form;
  * lognormal system sizes for the many-systems form.
"""
import numpy as np

SEED_BASE = 1209


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def uniform_cube(N: int, seed: int = SEED_BASE):
    """x ~ U[0,1)^3 (N x 3 float64), q ~ U[-1,1) (N float64)."""
    g = rng(seed)
    x = g.random((int(N), 3))
    q = g.random(int(N)) * 2.0 - 1.0
    return x, q


def plummer(N: int, seed: int = SEED_BASE + 2, rmax: float = 100.0):
    """Plummer sphere (a = 1) truncated at rmax, charges 1/N."""
    g = rng(seed)
    N = int(N)
    r = np.empty(0)
    while r.size < N:
        X = g.random(2 * (N - r.size) + 16)
        X = X[X > 0.0]
        rr = 1.0 / np.sqrt(X ** (-2.0 / 3.0) - 1.0)
        r = np.concatenate([r, rr[rr <= rmax]])
    r = r[:N]
    cz = g.random(N) * 2.0 - 1.0
    ph = g.random(N) * 2.0 * np.pi
    sz = np.sqrt(1.0 - cz * cz)
    x = np.stack([r * sz * np.cos(ph), r * sz * np.sin(ph), r * cz], axis=1)
    q = np.full(N, 1.0 / N)
    return x, q


def gaussian_charges(N: int, nrhs: int, seed: int = SEED_BASE + 3):
    """nrhs charge vectors q ~ N(0,1), shape (nrhs, N)."""
    return rng(seed).standard_normal((int(nrhs), int(N)))


def lognormal_sizes(nsys: int, lo: int = 1000, hi: int = 200000, seed: int = SEED_BASE + 3):
    """System sizes clamp(round(exp(N(ln sqrt(lo*hi), s^2))), lo, hi), +-2 s spanning [lo, hi]."""
    g = rng(seed)
    mu = 0.5 * (np.log(lo) + np.log(hi))
    s = 0.25 * (np.log(hi) - np.log(lo))
    n = np.rint(np.exp(g.normal(mu, s, int(nsys))))
    return np.clip(n, lo, hi).astype(np.int64)


def sample_targets(N: int, count: int = 4096):
    """Every (N // count)-th target of the original order (at most `count`)."""
    step = max(1, int(N) // int(count))
    return np.arange(0, int(N), step, dtype=np.int64)[:count]
