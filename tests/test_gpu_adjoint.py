"""GPU adjoint (fmm_backward) against the oracle's adjoint.

Bar: dL/dq and dL/dx within 1e-5 relative L2 of the FP64 oracle FMM adjoint at
the same P, theta, ncrit (same tree and lists); against the O(N^2) FP64
adjoint of the direct sum, within the oracle FMM's own error.  The autograd
wrapper gives the same numbers as the C ABI call, and the energy identities
dE/dq = phi, dE/dx = q grad hold to FP32 rounding.
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
    """Largest per-target error, each over rms(reference) + |reference at that
    target| (per-target vector norms for gradients): a bound on localised errors
    that the L2 norm can hide.  The |reference| term admits the FP32 rounding of
    a target's own largest terms (a close neighbour), which scales with them."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.abs(a - b) if a.ndim == 1 else np.linalg.norm(a - b, axis=-1)
    r = np.abs(b) if b.ndim == 1 else np.linalg.norm(b, axis=-1)
    return float(np.max(d / (np.sqrt(np.mean(r * r)) + r)))


def upstream(N, seed):
    g = inputs.rng(seed)
    return g.standard_normal(N).astype(np.float32), g.standard_normal((N, 3)).astype(np.float32)


def gpu_backward(torch, x, q32, a, b, P, theta, ncrit, kahan=False, hybrid=None):
    from paper_1209_3516_gb300 import fmm
    N = x.shape[0]
    h = fmm.FMM(N, P, theta, ncrit, kahan=kahan, hybrid=hybrid)
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    h.evaluate(torch.from_numpy(q32).cuda(), x=xd)
    ad = torch.from_numpy(a).cuda() if a is not None else None
    bd = torch.from_numpy(np.ascontiguousarray(b)).cuda() if b is not None else None
    dq, dx = h.backward(ad, bd)
    torch.cuda.synchronize()
    return h, dq.cpu().numpy(), dx.cpu().numpy()


CASES = [
    # N, P, theta, ncrit, kind
    (8192, 4, 0.4, 64, "u"),
    (16384, 6, 0.4, 64, "u"),
    (5001, 8, 0.45, 17, "u"),     # ragged: partial items and chunks
    (12000, 3, 0.5, 32, "u"),
    (20000, 4, 0.4, 32, "p"),     # adaptive (Plummer) tree
]


@pytest.mark.parametrize("N,P,theta,ncrit,kind", CASES)
def test_backward_parity_with_oracle(torch_cuda, N, P, theta, ncrit, kind):
    x, q = inputs.uniform_cube(N, 3100 + N) if kind == "u" else inputs.plummer(N, 3101 + N)
    if kind == "p":
        q = inputs.rng(3102 + N).random(N) * 2 - 1
    q32 = q.astype(np.float32)
    a, b = upstream(N, 3200 + N)
    h, dq, dx = gpu_backward(torch_cuda, x, q32, a, b, P, theta, ncrit)
    ref = oracle.FMM(N, P, theta, ncrit).build(x)
    rq, rx = ref.backward(q32.astype(np.float64), a.astype(np.float64), b.astype(np.float64))
    assert rel_l2(dq, rq) <= TOL, rel_l2(dq, rq)
    assert peak_rel(dq, rq) <= 10 * TOL, peak_rel(dq, rq)
    assert rel_l2(dx, rx) <= TOL, rel_l2(dx, rx)
    assert peak_rel(dx, rx) <= 10 * TOL, peak_rel(dx, rx)
    h.close()


def test_backward_against_direct_adjoint(torch_cuda):
    # the differentiated workload's check size: N = 8,192, P = 6, theta = 0.4
    N, P, theta = 8192, 6, 0.4
    x, q = inputs.uniform_cube(N, 3300)
    q32 = q.astype(np.float32)
    a, b = upstream(N, 3301)
    h, dq, dx = gpu_backward(torch_cuda, x, q32, a, b, P, theta, 64)
    q64, a64, b64 = q32.astype(np.float64), a.astype(np.float64), b.astype(np.float64)
    dq_d, dx_d = oracle.direct_backward(x, q64, a64, b64)
    oq, ox = oracle.FMM(N, P, theta, 64).build(x).backward(q64, a64, b64)
    e_gpu = (rel_l2(dq, dq_d), rel_l2(dx, dx_d))
    e_orc = (rel_l2(oq, dq_d), rel_l2(ox, dx_d))
    print("adjoint error vs direct: gpu dq %.2e dx %.2e, oracle FMM dq %.2e dx %.2e" % (e_gpu + e_orc))
    assert e_gpu[0] <= e_orc[0] * 1.05 + 2 * TOL
    assert e_gpu[1] <= e_orc[1] * 1.05 + 2 * TOL
    assert e_gpu[0] <= 1e-4 and e_gpu[1] <= 1e-4
    h.close()


def test_backward_theta_zero_is_direct_adjoint(torch_cuda):
    N = 6000
    x, q = inputs.uniform_cube(N, 3400)
    q32 = q.astype(np.float32)
    a, b = upstream(N, 3401)
    h, dq, dx = gpu_backward(torch_cuda, x, q32, a, b, 4, 0.0, 64)
    rq, rx = oracle.direct_backward(x, q32.astype(np.float64), a.astype(np.float64), b.astype(np.float64))
    assert rel_l2(dq, rq) <= TOL and rel_l2(dx, rx) <= TOL
    assert peak_rel(dq, rq) <= 10 * TOL and peak_rel(dx, rx) <= 10 * TOL
    h.close()


@pytest.mark.parametrize("which", ["dphi", "dgrad"])
def test_backward_one_upstream_gradient(torch_cuda, which):
    N = 7000
    x, q = inputs.uniform_cube(N, 3500)
    q32 = q.astype(np.float32)
    a, b = upstream(N, 3501)
    a_, b_ = (a, None) if which == "dphi" else (None, b)
    h, dq, dx = gpu_backward(torch_cuda, x, q32, a_, b_, 5, 0.4, 32)
    rq, rx = oracle.FMM(N, 5, 0.4, 32).build(x).backward(
        q32.astype(np.float64), None if a_ is None else a.astype(np.float64), None if b_ is None else b.astype(np.float64))
    assert rel_l2(dq, rq) <= TOL and rel_l2(dx, rx) <= TOL
    assert peak_rel(dq, rq) <= 10 * TOL and peak_rel(dx, rx) <= 10 * TOL
    h.close()


def test_backward_outputs_optional_and_repeatable(torch_cuda):
    torch = torch_cuda
    from paper_1209_3516_gb300 import fmm
    N = 4000
    x, q = inputs.uniform_cube(N, 3600)
    a, b = upstream(N, 3601)
    h = fmm.FMM(N, 4, 0.4, 32)
    with pytest.raises(fmm.FMMError) as e:
        h.backward(torch.from_numpy(a).cuda(), None)
    assert e.value.code == fmm.FMM_ERR_STATE
    h.evaluate(torch.from_numpy(q.astype(np.float32)).cuda(), x=torch.from_numpy(x).cuda())
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    dq1, dx1 = h.backward(ad, bd)
    dq2, _ = h.backward(ad, bd, want_dx=False)
    _, dx3 = h.backward(ad, bd, want_dq=False)
    assert torch.equal(dq1, dq2) and torch.equal(dx1, dx3)
    with pytest.raises(fmm.FMMError) as e:
        h.backward(ad, bd, want_dq=False, want_dx=False)
    assert e.value.code == fmm.FMM_ERR_ARG
    h.close()


def test_backward_with_compensated_forward(torch_cuda):
    # a handle created for compensated P2P (work items of <= 8 targets)
    N = 9000
    x, q = inputs.plummer(N, 3700)
    q32 = q.astype(np.float32)
    a, b = upstream(N, 3701)
    h, dq, dx = gpu_backward(torch_cuda, x, q32, a, b, 4, 0.4, 64, kahan=True)
    rq, rx = oracle.FMM(N, 4, 0.4, 64).build(x).backward(q32.astype(np.float64), a.astype(np.float64),
                                                          b.astype(np.float64))
    assert rel_l2(dq, rq) <= TOL and rel_l2(dx, rx) <= TOL
    assert peak_rel(dq, rq) <= 10 * TOL and peak_rel(dx, rx) <= 10 * TOL
    h.close()


def test_backward_with_hybrid_lists(torch_cuda):
    # the adjoint runs over whatever lists the traversal made, here the M2L / P2P hybrid's
    N = 12000
    x, q = inputs.uniform_cube(N, 3750)
    q32 = q.astype(np.float32)
    a, b = upstream(N, 3751)
    h, dq, dx = gpu_backward(torch_cuda, x, q32, a, b, 6, 0.5, 32, hybrid=0)
    rq, rx = oracle.FMM(N, 6, 0.5, 32, hybrid_min_pairs=0).build(x).backward(
        q32.astype(np.float64), a.astype(np.float64), b.astype(np.float64))
    assert rel_l2(dq, rq) <= TOL and rel_l2(dx, rx) <= TOL
    assert peak_rel(dq, rq) <= 10 * TOL and peak_rel(dx, rx) <= 10 * TOL
    h.close()


def test_autograd_general_loss(torch_cuda):
    torch = torch_cuda
    from paper_1209_3516_gb300 import autograd, fmm
    N, P, theta = 10000, 6, 0.4
    x, q = inputs.uniform_cube(N, 3800)
    a, b = upstream(N, 3801)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    qt = torch.from_numpy(q.astype(np.float32)).cuda().requires_grad_(True)
    h = fmm.FMM(N, P, theta, 64)
    phi, grad = autograd.laplace_fmm(xt, qt, h)
    loss = (phi * torch.from_numpy(a).cuda()).sum() + (grad * torch.from_numpy(b).cuda()).sum()
    loss.backward()
    assert xt.grad.dtype == torch.float64 and qt.grad.dtype == torch.float32
    rq, rx = oracle.FMM(N, P, theta, 64).build(x).backward(q.astype(np.float32).astype(np.float64),
                                                           a.astype(np.float64), b.astype(np.float64))
    assert rel_l2(qt.grad.cpu().numpy(), rq) <= TOL
    assert peak_rel(qt.grad.cpu().numpy(), rq) <= 10 * TOL, peak_rel(qt.grad.cpu().numpy(), rq)
    assert rel_l2(xt.grad.cpu().numpy(), rx) <= TOL
    assert peak_rel(xt.grad.cpu().numpy(), rx) <= 10 * TOL, peak_rel(xt.grad.cpu().numpy(), rx)
    # a second evaluation on the same handle invalidates the first graph
    phi2, _ = autograd.laplace_fmm(xt, qt, h)
    phi3, _ = autograd.laplace_fmm(xt, qt, h)
    with pytest.raises(RuntimeError, match="evaluated again"):
        phi2.sum().backward()
    h.close()


def test_autograd_energy_identities(torch_cuda):
    # E = 1/2 sum q phi: dE/dq = phi and dE/dx = q grad (symmetric kernel), here
    # with phi, grad from the forward kernels and the gradients from the adjoint ones
    torch = torch_cuda
    from paper_1209_3516_gb300 import autograd, fmm
    N = 16384
    x, q = inputs.uniform_cube(N, 3900)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    qt = torch.from_numpy(q.astype(np.float32)).cuda().requires_grad_(True)
    h = fmm.FMM(N, 6, 0.4, 64)
    phi, grad = autograd.laplace_fmm(xt, qt, h)
    E = 0.5 * (qt.double() * phi.double()).sum()
    E.backward()
    phi_n = phi.detach().cpu().numpy().astype(np.float64)
    g_n = grad.detach().cpu().numpy().astype(np.float64)
    assert rel_l2(qt.grad.cpu().numpy(), phi_n) <= TOL
    assert peak_rel(qt.grad.cpu().numpy(), phi_n) <= 10 * TOL, peak_rel(qt.grad.cpu().numpy(), phi_n)
    assert rel_l2(xt.grad.cpu().numpy(), q.astype(np.float32)[:, None] * g_n) <= TOL
    assert peak_rel(xt.grad.cpu().numpy(), q.astype(np.float32)[:, None] * g_n) <= 10 * TOL, peak_rel(xt.grad.cpu().numpy(), q.astype(np.float32)[:, None] * g_n)
    h.close()


@pytest.mark.slow
def test_full_size_differentiated_262k(torch_cuda):
    # the differentiated workload: N = 262,144, P = 6, theta = 0.4; sampled parity
    N, P, theta, ncrit = 262144, 6, 0.4, 64
    x, q = inputs.uniform_cube(N, inputs.SEED_BASE + 5)
    q32 = q.astype(np.float32)
    a, b = upstream(N, inputs.SEED_BASE + 6)
    h, dq, dx = gpu_backward(torch_cuda, x, q32, a, b, P, theta, ncrit)
    t = inputs.sample_targets(N, 4096)
    q64, a64, b64 = q32.astype(np.float64), a.astype(np.float64), b.astype(np.float64)
    rq, rx = oracle.FMM(N, P, theta, ncrit).build(x).backward(q64, a64, b64, targets=t)
    assert rel_l2(dq[t], rq) <= TOL
    assert peak_rel(dq[t], rq) <= 10 * TOL, peak_rel(dq[t], rq)
    assert rel_l2(dx[t], rx) <= TOL
    assert peak_rel(dx[t], rx) <= 10 * TOL, peak_rel(dx[t], rx)
    dq_d, dx_d = oracle.direct_backward(x, q64, a64, b64, targets=t)
    st = h.stats()
    print("N=262144 P=6 theta=0.4 adjoint: err vs direct dq %.2e dx %.2e; backward %.3f ms, evaluate %.3f ms"
          % (rel_l2(dq[t], dq_d), rel_l2(dx[t], dx_d), st["ms_backward"], st["ms_evaluate"]))
    h.close()
