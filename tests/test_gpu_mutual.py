"""Mutual (Newton's third law) near field, FMM_FLAG_MUTUAL, on the GPU.

Each unordered pair of leaves of the P2P list is evaluated once and applied to
both leaves (the falcON heritage the paper cites in Sec. 2); the lists are the
same as Algorithm 4's, so the results must match the oracle FMM at the same
tolerance as the one-sided path, match that path to rounding, reproduce the
direct sum at theta = 0 and keep the total force balanced.
"""
import numpy as np
import pytest

import oracle
from paper_1209_3516_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_1209_3516_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def peak_rel(a, b):
    """Largest per-target error over rms(reference) + |reference at that target|."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.abs(a - b) if a.ndim == 1 else np.linalg.norm(a - b, axis=-1)
    r = np.abs(b) if b.ndim == 1 else np.linalg.norm(b, axis=-1)
    return float(np.max(d / (np.sqrt(np.mean(r * r)) + r)))


def run(torch, x, q, P, theta, ncrit, mutual, hybrid=None):
    from paper_1209_3516_gb300 import fmm
    N = x.shape[0]
    h = fmm.FMM(N, P, theta, ncrit, mutual=mutual, hybrid=hybrid)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    qd = torch.from_numpy(q.astype(np.float32)).cuda()
    h.build(xd)
    phi, grad = h.evaluate(qd)
    torch.cuda.synchronize()
    out = phi.cpu().numpy(), grad.cpu().numpy()
    h.close()
    return out


CASES = [
    (16384, 4, 0.4, 64, "u"),
    (16384, 8, 0.5, 64, "u"),
    (33333, 4, 0.45, 32, "u"),    # ragged: partial items and chunks
    (20000, 4, 0.4, 32, "p"),     # adaptive (Plummer) tree
    (9000, 6, 0.5, 8, "p"),
]


@pytest.mark.parametrize("N,P,theta,ncrit,kind", CASES)
def test_mutual_parity_with_oracle(torch_cuda, N, P, theta, ncrit, kind):
    x, q = inputs.uniform_cube(N, 1209 + N) if kind == "u" else inputs.plummer(N, 1211 + N)
    if kind == "p":
        q = inputs.rng(7 + N).random(N) * 2 - 1
    q32 = q.astype(np.float32).astype(np.float64)
    phi, grad = run(torch_cuda, x, q32, P, theta, ncrit, mutual=True)
    pr, gr = oracle.FMM(N, P, theta, ncrit).build(x).evaluate(q32)
    assert rel_l2(phi, pr) <= TOL and rel_l2(grad, gr) <= TOL, (rel_l2(phi, pr), rel_l2(grad, gr))
    assert peak_rel(phi, pr) <= 10 * TOL and peak_rel(grad, gr) <= 10 * TOL, (peak_rel(phi, pr), peak_rel(grad, gr))
    # the one-sided path on the same inputs: equal to FP32 rounding
    p1, g1 = run(torch_cuda, x, q32, P, theta, ncrit, mutual=False)
    assert rel_l2(phi, p1) <= 1e-6 and rel_l2(grad, g1) <= 1e-6, (rel_l2(phi, p1), rel_l2(grad, g1))


def test_mutual_theta_zero_direct_sum_and_force_balance(torch_cuda):
    # every pair of leaves goes to P2P: the direct sum, and sum_i q_i grad phi_i = 0
    N = 12000
    x, q = inputs.uniform_cube(N, 77)
    q32 = q.astype(np.float32).astype(np.float64)
    phi, grad = run(torch_cuda, x, q32, 4, 0.0, 64, mutual=True)
    pd, gd = oracle.direct(x, q32)
    assert rel_l2(phi, pd) <= TOL and rel_l2(grad, gd) <= TOL
    f = q32[:, None] * grad.astype(np.float64)
    balance = np.linalg.norm(f.sum(axis=0)) / np.abs(f).sum()
    assert balance < 1e-6, balance


def test_mutual_with_hybrid_leaves(torch_cuda):
    # the M2L / P2P hybrid keeps the P2P list symmetric: the mutual pass still applies
    N, P, theta, ncrit = 20000, 6, 0.5, 32
    x, q = inputs.uniform_cube(N, 4040)
    q32 = q.astype(np.float32).astype(np.float64)
    phi, grad = run(torch_cuda, x, q32, P, theta, ncrit, mutual=True, hybrid=256)
    ref = oracle.FMM(N, P, theta, ncrit, hybrid_min_pairs=256).build(x)
    pr, gr = ref.evaluate(q32)
    assert rel_l2(phi, pr) <= TOL and rel_l2(grad, gr) <= TOL


def test_mutual_full_size_sampled(torch_cuda):
    # the benchmark workload (N = 1,048,576, P = 8, theta = 0.5) against the FP64 direct sum on 4,096 targets
    N, P, theta, ncrit = 1048576, 8, 0.5, 64
    x, q = inputs.uniform_cube(N, inputs.SEED_BASE + 1)
    q32 = q.astype(np.float32).astype(np.float64)
    phi, grad = run(torch_cuda, x, q32, P, theta, ncrit, mutual=True)
    t = np.arange(0, N, 256)
    pd, gd = oracle.direct(x, q32, targets=t)
    assert rel_l2(phi[t], pd) <= 1e-4 and rel_l2(grad[t], gd) <= 1e-4, (rel_l2(phi[t], pd), rel_l2(grad[t], gd))
