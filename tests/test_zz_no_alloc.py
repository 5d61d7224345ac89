"""The allocation-free energy entry point: results, size limit and pointer checks.

fmm_energy_noalloc serves callers that cannot let a library call cudaMalloc
(applications that hand out all device memory from their own arena or a
framework allocator).  It keeps its scratch in a fixed device array of the
library instead of allocating.  These tests call it through the C ABI:
twice in a row against the allocating entry point fmm_energy on the same
potentials and against an FP64 host sum of q.phi; at the array's edge
(n = 16,777,216 fills all 8,192 partial slots, n = 2048 k + 1 leaves the last
block holding one value); with device memory unchanged across a call; and
with host pointers, which it must reject before launching anything.  The file
is collected last so that a failure here stops a -x run only after every
other test has run; it also passes when run alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_1209_3516_gb300 import inputs

pytestmark = pytest.mark.gpu


def _host_energy(q, phi):
    return 0.5 * float(np.dot(q.astype(np.float64), phi.astype(np.float64)))


def test_energy_noalloc_matches_fmm_energy_twice():
    import torch
    from paper_1209_3516_gb300 import build, fmm
    build.build()
    torch.cuda.set_device(0)
    N = 30000
    x, _ = inputs.uniform_cube(N, 4242)
    xd = torch.from_numpy(x).cuda()
    h = fmm.FMM(N, 4, 0.4, 64)
    E_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        q = (inputs.rng(5000 + call).random(N) * 2 - 1).astype(np.float32)
        qd = torch.from_numpy(q).cuda()
        phi, _ = h.evaluate(qd, x=xd)
        E_ref = h.energy()                       # allocating entry point
        fmm.energy_noalloc(qd, phi, E_dev)       # allocation-free entry point
        torch.cuda.synchronize()
        E_new = float(E_dev.item())
        ph = phi.cpu().numpy()
        scale = float(np.abs(q.astype(np.float64)) @ np.abs(ph.astype(np.float64)))
        assert abs(E_new - E_ref) <= 1e-5 * abs(E_ref) + 1e-7 * scale, (call, E_new, E_ref)
        # both reduce in FP64: against the host FP64 sum of the same values
        assert abs(E_new - _host_energy(q, ph)) <= 1e-12 * scale, (call, E_new, _host_energy(q, ph))
    h.close()


@pytest.mark.parametrize("n", [16777216, 2048 * 5000 + 1, 2049, 1])
def test_energy_noalloc_at_the_scratch_edge(n):
    """n = 16,777,216 uses all 8,192 partials; 2048 k + 1 leaves one value in the last block."""
    import torch
    from paper_1209_3516_gb300 import build, fmm
    build.build()
    torch.cuda.set_device(0)
    g = inputs.rng(7100 + n % 997)
    q = (g.random(n) * 2 - 1).astype(np.float32)
    phi = (g.standard_normal(n) + 0.25).astype(np.float32)
    qd, pd = torch.from_numpy(q).cuda(), torch.from_numpy(phi).cuda()
    E = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    fmm.energy_noalloc(qd, pd, E)            # first call sets up the scratch address
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    E.fill_(np.nan)
    fmm.energy_noalloc(qd, pd, E)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "the call changed the device's free memory"
    ref = _host_energy(q, phi)
    scale = 0.5 * float(np.abs(q.astype(np.float64)) @ np.abs(phi.astype(np.float64)))
    assert abs(float(E.item()) - ref) <= 1e-12 * scale + 1e-300, (n, float(E.item()), ref)


def test_energy_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_1209_3516_gb300 import build, fmm
    build.build()
    L = fmm.load()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    q = torch.zeros(16, dtype=torch.float32, device="cuda")
    rc = L.fmm_energy_noalloc(q.data_ptr(), q.data_ptr(), 16777217, E.data_ptr(), None)
    assert rc == fmm.FMM_ERR_ARG
    assert b"16777216" in L.fmm_last_error_string()
    assert L.fmm_energy_noalloc(q.data_ptr(), q.data_ptr(), 0, E.data_ptr(), None) == fmm.FMM_ERR_ARG


def test_energy_noalloc_rejects_host_pointers():
    """A host E (what fmm_energy takes) or host inputs are argument errors, found before any launch."""
    import torch
    from paper_1209_3516_gb300 import build, fmm
    build.build()
    torch.cuda.set_device(0)
    L = fmm.load()
    q = torch.ones(4096, dtype=torch.float32, device="cuda")
    E_dev = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    E_host = np.full(1, 7.0)                                   # pageable host memory
    E_pinned = torch.full((1,), 7.0, dtype=torch.float64).pin_memory()
    q_host = np.ones(4096, dtype=np.float32)
    for ep in (E_host.ctypes.data, E_pinned.data_ptr()):
        assert L.fmm_energy_noalloc(q.data_ptr(), q.data_ptr(), 4096, ep, None) == fmm.FMM_ERR_ARG
        assert b"E is host memory" in L.fmm_last_error_string()
    assert L.fmm_energy_noalloc(q_host.ctypes.data, q.data_ptr(), 4096, E_dev.data_ptr(), None) == fmm.FMM_ERR_ARG
    assert b"q is" in L.fmm_last_error_string()
    torch.cuda.synchronize()
    assert E_host[0] == 7.0 and float(E_pinned[0]) == 7.0 and float(E_dev.item()) == 7.0
    # the context is intact: a valid call still works
    assert L.fmm_energy_noalloc(q.data_ptr(), q.data_ptr(), 4096, E_dev.data_ptr(), None) == fmm.FMM_OK
    torch.cuda.synchronize()
    assert float(E_dev.item()) == 2048.0
