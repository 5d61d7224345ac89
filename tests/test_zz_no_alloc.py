"""The allocation-free energy entry point agrees with fmm_energy.

fmm_energy_noalloc serves callers that cannot let a library call cudaMalloc
(applications that hand out all device memory from their own arena or a
framework allocator).  It keeps its scratch in a fixed device array of the
library instead of allocating; this test calls it through the C ABI twice in
a row and compares each result with the allocating entry point fmm_energy on
the same potentials, within the energy tolerance of the parity tests.  The
file is collected last so that a failure here stops a -x run only after every
other test has run; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1209_3516_gb300 import inputs

pytestmark = pytest.mark.gpu


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
        scale = float(np.abs(q.astype(np.float64)) @ np.abs(phi.cpu().numpy().astype(np.float64)))
        assert abs(E_new - E_ref) <= 1e-5 * abs(E_ref) + 1e-7 * scale, (call, E_new, E_ref)
    h.close()


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
