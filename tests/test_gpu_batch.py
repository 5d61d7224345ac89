"""Many charge vectors on one geometry (fmm_evaluate_batch) against the oracle.

The batched path runs the far field in FP32 and the P2P as a tensor-core
product with BF16 high/low splits of the kernel matrix and the charges (three
MMAs, FP32 accumulation).  BF16 keeps 8 significant bits (unit roundoff
2^-8), so v = hi + lo holds v to 2^-16 relative, and the dropped low*low
product and the two low-part roundings leave at most about 3 * 2^-16
(4.6e-5) of each pair term; potentials of zero-mean charges cancel, so the
relative L2 error of a whole vector can sit a little above that.  The bar is
the batched workload's stated accuracy, 1e-4 relative L2 per vector against
the FP64 oracle FMM at the same P, theta, ncrit, and every vector is checked.
"""
import numpy as np
import pytest

import oracle
from paper_1209_3516_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL_B = 1e-4


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
    """Largest per-target error, each over rms(reference) + |reference at that
    target| (per-target vector norms for gradients): a bound on localised errors
    that the L2 norm can hide.  The |reference| term admits the FP32 rounding of
    a target's own largest terms (a close neighbour), which scales with them."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.abs(a - b) if a.ndim == 1 else np.linalg.norm(a - b, axis=-1)
    r = np.abs(b) if b.ndim == 1 else np.linalg.norm(b, axis=-1)
    return float(np.max(d / (np.sqrt(np.mean(r * r)) + r)))


def run_batch(torch, x, Q, P, theta, ncrit):
    from paper_1209_3516_gb300 import fmm
    N = x.shape[0]
    h = fmm.FMM(N, P, theta, ncrit)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    qd = torch.from_numpy(np.ascontiguousarray(Q, dtype=np.float32)).cuda()
    phi, grad = h.evaluate_batch(qd, x=xd)
    torch.cuda.synchronize()
    return h, phi.cpu().numpy(), grad.cpu().numpy()


CASES = [
    # N, P, theta, ncrit, nrhs, kind
    (16384, 4, 0.4, 64, 32, "u"),
    (16384, 8, 0.5, 64, 32, "u"),
    (9001, 6, 0.45, 23, 7, "u"),      # ragged N, partial batch
    (20000, 4, 0.4, 32, 32, "p"),     # adaptive tree
    (3000, 3, 0.5, 16, 1, "u"),
]


@pytest.mark.parametrize("N,P,theta,ncrit,nrhs,kind", CASES)
def test_batch_parity_with_oracle(torch_cuda, N, P, theta, ncrit, nrhs, kind):
    x, _ = inputs.uniform_cube(N, 4100 + N) if kind == "u" else inputs.plummer(N, 4101 + N)
    Q = inputs.gaussian_charges(N, nrhs, 4200 + N).astype(np.float32)
    h, phi, grad = run_batch(torch_cuda, x, Q, P, theta, ncrit)
    assert phi.shape == (nrhs, N) and grad.shape == (nrhs, N, 3)
    ref = oracle.FMM(N, P, theta, ncrit).build(x)
    worst = (0.0, 0.0)
    for r in range(nrhs):
        pr, gr = ref.evaluate(Q[r].astype(np.float64))
        e = (rel_l2(phi[r], pr), rel_l2(grad[r], gr))
        worst = (max(worst[0], e[0]), max(worst[1], e[1]))
        assert e[0] <= TOL_B and e[1] <= TOL_B, (r, e)
        pk = (peak_rel(phi[r], pr), peak_rel(grad[r], gr))
        assert pk[0] <= 10 * TOL_B and pk[1] <= 10 * TOL_B, (r, pk)
    print("batch N=%d P=%d nrhs=%d: worst rel err phi %.2e grad %.2e" % (N, P, nrhs, worst[0], worst[1]))
    h.close()


def test_batch_matches_single_vector_path(torch_cuda):
    torch = torch_cuda
    N, nrhs = 12000, 5
    x, _ = inputs.uniform_cube(N, 4300)
    Q = inputs.gaussian_charges(N, nrhs, 4301).astype(np.float32)
    h, phi, grad = run_batch(torch, x, Q, 5, 0.4, 32)
    for r in range(nrhs):
        p1, g1 = h.evaluate(torch.from_numpy(Q[r]).cuda())
        assert rel_l2(phi[r], p1.cpu().numpy().astype(np.float64)) <= TOL_B
        assert rel_l2(grad[r], g1.cpu().numpy().astype(np.float64)) <= TOL_B
    h.close()


def test_batch_theta_zero_is_the_direct_sum(torch_cuda):
    N, nrhs = 6000, 4
    x, _ = inputs.uniform_cube(N, 4400)
    Q = inputs.gaussian_charges(N, nrhs, 4401).astype(np.float32)
    h, phi, grad = run_batch(torch_cuda, x, Q, 4, 0.0, 64)
    for r in range(nrhs):
        pd, gd = oracle.direct(x, Q[r].astype(np.float64))
        assert rel_l2(phi[r], pd) <= TOL_B and rel_l2(grad[r], gd) <= TOL_B
        assert peak_rel(phi[r], pd) <= 10 * TOL_B and peak_rel(grad[r], gd) <= 10 * TOL_B
    h.close()


def test_batch_argument_checks(torch_cuda):
    torch = torch_cuda
    from paper_1209_3516_gb300 import fmm
    N = 1000
    x, _ = inputs.uniform_cube(N, 4500)
    h = fmm.FMM(N, 4, 0.4, 64)
    xd = torch.from_numpy(x).cuda()
    for nrhs in (0, 33):
        q = torch.zeros(max(nrhs, 1), N, dtype=torch.float32, device="cuda")
        with pytest.raises(fmm.FMMError) as e:
            from paper_1209_3516_gb300.fmm import load, _check
            _check(load().fmm_evaluate_batch(h._h, xd.data_ptr(), q.data_ptr(), nrhs, q.data_ptr(), None))
        assert e.value.code == fmm.FMM_ERR_ARG
    h.close()


@pytest.mark.slow
def test_full_size_batched_1m(torch_cuda):
    # the batched workload: N = 1,048,576 uniform cube, 32 Gaussian charge vectors,
    # P = 8, theta = 0.5; every vector against the oracle FMM on a 4,096-target sample
    torch = torch_cuda
    N, P, theta, ncrit, nrhs = 1048576, 8, 0.5, 64, 32
    x, _ = inputs.uniform_cube(N, inputs.SEED_BASE + 1)
    Q = inputs.gaussian_charges(N, nrhs, inputs.SEED_BASE + 3).astype(np.float32)
    h, phi, grad = run_batch(torch, x, Q, P, theta, ncrit)
    ref = oracle.FMM(N, P, theta, ncrit).build(x)
    t = inputs.sample_targets(N, 4096)
    worst = [0.0, 0.0, 0.0]
    for r in range(nrhs):
        pr, gr = ref.evaluate(Q[r].astype(np.float64), t)
        e = (rel_l2(phi[r][t], pr), rel_l2(grad[r][t], gr))
        worst[0], worst[1] = max(worst[0], e[0]), max(worst[1], e[1])
        assert e[0] <= TOL_B and e[1] <= TOL_B, (r, e)
        if r < 2:
            pd, gd = oracle.direct(x, Q[r].astype(np.float64), t)
            worst[2] = max(worst[2], rel_l2(phi[r][t], pd), rel_l2(grad[r][t], gd))
    print("batched N=1M P=8 theta=0.5 x32: worst vs oracle FMM phi %.2e grad %.2e; vs direct %.2e; %.3f ms"
          % (worst[0], worst[1], worst[2], h.stats()["ms_batch"]))
    assert worst[2] <= 1e-4
    h.close()
