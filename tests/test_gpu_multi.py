"""Many independent systems in one evaluation (fmm_multi_*) against the oracle.

The merged problem runs the same kernels as one system, so the bar is the
plain FP32 path's: 1e-5 relative L2 per system against the FP64 oracle FMM of
that system alone (its own tree, lists and normalisation).
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


def systems(sizes, seed, plummer_every=0):
    xs, qs = [], []
    for k, n in enumerate(sizes):
        if plummer_every and k % plummer_every == plummer_every - 1:
            x, _ = inputs.plummer(n, seed + k)
            q = inputs.rng(seed + 1000 + k).random(n) * 2 - 1
        else:
            x, q = inputs.uniform_cube(n, seed + k)
        xs.append(x)
        qs.append(q.astype(np.float32))
    return xs, qs


def run_multi(torch, xs, qs, P, theta, ncrit, hybrid=None, config=None):
    from paper_1209_3516_gb300 import fmm
    sizes = [x.shape[0] for x in xs]
    m = fmm.MultiFMM(sizes, P, theta, ncrit, hybrid=hybrid)
    if config is not None:
        m.set_config(*config)
    m.build(torch.from_numpy(np.concatenate(xs)).cuda())
    q = torch.from_numpy(np.concatenate(qs)).cuda()
    phi, grad = m.evaluate(q)
    torch.cuda.synchronize()
    return m, q, phi, grad


@pytest.mark.parametrize("P,theta,ncrit", [(4, 0.4, 64), (8, 0.5, 32), (3, 0.5, 16)])
def test_multi_parity_with_oracle(torch_cuda, P, theta, ncrit):
    sizes = [3000, 17, 1, 12000, 800, 5001, 64, 20000]
    xs, qs = systems(sizes, 5100 + P, plummer_every=3)
    m, q, phi, grad = run_multi(torch_cuda, xs, qs, P, theta, ncrit)
    phi, grad = phi.cpu().numpy(), grad.cpu().numpy()
    off = 0
    for x, qq in zip(xs, qs):
        n = x.shape[0]
        pr, gr = oracle.FMM(n, P, theta, ncrit).build(x).evaluate(qq.astype(np.float64))
        if n == 1:
            assert phi[off] == 0.0 and np.all(grad[off] == 0.0)
        else:
            assert rel_l2(phi[off:off + n], pr) <= TOL, (n, rel_l2(phi[off:off + n], pr))
            assert peak_rel(phi[off:off + n], pr) <= 10 * TOL, peak_rel(phi[off:off + n], pr)
            assert rel_l2(grad[off:off + n], gr) <= TOL, (n, rel_l2(grad[off:off + n], gr))
            assert peak_rel(grad[off:off + n], gr) <= 10 * TOL, peak_rel(grad[off:off + n], gr)
        off += n
    info = m.info()
    assert info["nsys"] == len(sizes) and info["n_total"] == sum(sizes)
    assert info["graph_nodes"] > 0 and info["p2p_targets_per_item"] in (8, 16)
    m.close()


def test_multi_graph_replay_and_recapture(torch_cuda):
    torch = torch_cuda
    sizes = [4000, 2500, 9000]
    xs, qs = systems(sizes, 5200)
    m, q, phi1, grad1 = run_multi(torch, xs, qs, 5, 0.4, 32)
    p1, g1 = phi1.clone(), grad1.clone()
    phi2, grad2 = m.evaluate(q, phi=phi1, grad=grad1)   # same pointers: graph replay
    torch.cuda.synchronize()
    if m.info()["mutual"]:   # float reductions of the mutual near field: equal to rounding
        assert rel_l2(phi2.cpu().numpy(), p1.cpu().numpy().astype(np.float64)) <= 1e-6
        assert rel_l2(grad2.cpu().numpy(), g1.cpu().numpy().astype(np.float64)) <= 1e-6
    else:                    # one-sided: bitwise the same
        assert torch.equal(phi2, p1) and torch.equal(grad2, g1)
    q2 = q * 2.0                                       # new pointer: new capture, linear in q
    phi3, grad3 = m.evaluate(q2)
    torch.cuda.synchronize()
    assert rel_l2(phi3.cpu().numpy(), 2 * p1.cpu().numpy().astype(np.float64)) <= 1e-6
    assert rel_l2(grad3.cpu().numpy(), 2 * g1.cpu().numpy().astype(np.float64)) <= 1e-6
    # the same systems through plain handles agree to rounding
    from paper_1209_3516_gb300 import fmm
    off = 0
    for x, qq in zip(xs, qs):
        n = x.shape[0]
        h = fmm.FMM(n, 5, 0.4, 32)
        pp, gg = h.evaluate(torch.from_numpy(qq).cuda(), x=torch.from_numpy(x).cuda())
        assert rel_l2(p1[off:off + n].cpu().numpy(), pp.cpu().numpy().astype(np.float64)) <= 1e-6
        assert rel_l2(g1[off:off + n].cpu().numpy(), gg.cpu().numpy().astype(np.float64)) <= 1e-6
        h.close()
        off += n
    m.close()


@pytest.mark.slow
def test_multi_64_lognormal_systems(torch_cuda):
    # the many-systems workload: 64 systems, N lognormal in [1000, 200000], uniform
    # cube, charges U[-1,1), P = 8, theta = 0.5; every system sampled against the oracle
    torch = torch_cuda
    sizes = [int(n) for n in inputs.lognormal_sizes(64)]
    xs, qs = systems(sizes, inputs.SEED_BASE + 10)
    m, q, phi, grad = run_multi(torch, xs, qs, 8, 0.5, 64)
    phi, grad = phi.cpu().numpy(), grad.cpu().numpy()
    off, worst = 0, (0.0, 0.0)
    for x, qq in zip(xs, qs):
        n = x.shape[0]
        t = inputs.sample_targets(n, 512)
        pr, gr = oracle.FMM(n, 8, 0.5, 64).build(x).evaluate(qq.astype(np.float64), t)
        e = (rel_l2(phi[off + t], pr), rel_l2(grad[off + t], gr))
        worst = (max(worst[0], e[0]), max(worst[1], e[1]))
        assert e[0] <= TOL and e[1] <= TOL, (n, e)
        off += n
    info = m.info()
    print("64 systems, N total %d: worst phi %.2e grad %.2e; graph nodes %d; P2P items of %d targets "
          "(tuned %.3f / %.3f ms); replay %.3f ms" % (sum(sizes), worst[0], worst[1], info["graph_nodes"],
                                                     info["p2p_targets_per_item"], info["tune_ms"][0],
                                                     info["tune_ms"][1], info["ms_evaluate"]))
    m.close()


def test_multi_with_hybrid(torch_cuda):
    # the M2L / P2P hybrid applied to every system: each system against its own
    # oracle run with the same rule
    sizes = [6000, 300, 15000, 2500]
    xs, qs = systems(sizes, 5300, plummer_every=2)
    m, q, phi, grad = run_multi(torch_cuda, xs, qs, 8, 0.5, 32, hybrid=0)
    phi, grad = phi.cpu().numpy(), grad.cpu().numpy()
    off = 0
    for x, qq in zip(xs, qs):
        n = x.shape[0]
        pr, gr = oracle.FMM(n, 8, 0.5, 32, hybrid_min_pairs=0).build(x).evaluate(qq.astype(np.float64))
        assert rel_l2(phi[off:off + n], pr) <= TOL and rel_l2(grad[off:off + n], gr) <= TOL
        assert peak_rel(phi[off:off + n], pr) <= 10 * TOL and peak_rel(grad[off:off + n], gr) <= 10 * TOL
        off += n
    m.close()


@pytest.mark.parametrize("g,mutual", [(16, 0), (8, 0), (16, 1), (8, 1), (16, 2), (8, 2)])
def test_multi_every_tile_configuration(torch_cuda, g, mutual):
    # each configuration the autotuner may choose, pinned: every system against its oracle
    sizes = [5000, 40, 11000, 900, 3001]
    xs, qs = systems(sizes, 5400, plummer_every=2)
    m, q, phi, grad = run_multi(torch_cuda, xs, qs, 6, 0.45, 32, config=(g, mutual))
    info = m.info()
    assert info["p2p_targets_per_item"] == g and info["mutual"] == mutual
    assert all(t > 0 for t in info["tune_ms"])
    phi, grad = phi.cpu().numpy(), grad.cpu().numpy()
    off = 0
    for x, qq in zip(xs, qs):
        n = x.shape[0]
        pr, gr = oracle.FMM(n, 6, 0.45, 32).build(x).evaluate(qq.astype(np.float64))
        assert rel_l2(phi[off:off + n], pr) <= TOL and rel_l2(grad[off:off + n], gr) <= TOL, (n, g, mutual)
        assert peak_rel(phi[off:off + n], pr) <= 10 * TOL and peak_rel(grad[off:off + n], gr) <= 10 * TOL
        off += n
    m.close()
