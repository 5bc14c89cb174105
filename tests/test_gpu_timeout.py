"""Bounded device-side waits (MOR_ERR_TIMEOUT) without a GPU fault.

The reduced CG runs as one cooperative launch whose grid barriers wait with a budget
(mor_set_wait_budget).  The timeout path is exercised on a flag that nothing sets: the
wait must run out, the kernel return, the call report MOR_ERR_TIMEOUT, and the CUDA
context stay usable, which a reduced solve right after it shows.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mor():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2404_06260_gb300 import _build
    _build.build()
    from paper_2404_06260_gb300 import mor as m
    return m


def test_wait_on_an_unset_flag_times_out_and_the_context_survives(mor):
    import time
    t0 = time.perf_counter()
    assert mor.debug_wait_timeout(0.01) is True
    assert time.perf_counter() - t0 < 5.0
    assert mor._lib.mor_debug_wait_timeout(0.001, None) == -1   # argument check
    # the context is still usable: a reduced solve with the default budget converges
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    b = mor.Bases(sd, mor.basis_opts(rank=p["rank"], oversample=p["oversample"],
                                     seed=p["seed"], precision="fp64", cg_rtol=1e-13))
    r = mor.Reduced(sd, b)
    mor.set_wait_budget(1.0)
    x, info = r.solve(rtol=1e-13)
    assert info["converged"]
    K = r.dense()
    xd = np.linalg.solve(K, b.bt().ravel())
    assert np.allclose(x.cpu().numpy(), xd, rtol=0, atol=1e-10 * np.abs(xd).max())


def test_wait_budget_argument_checks(mor):
    with pytest.raises(mor.MorError):
        mor.set_wait_budget(-1.0)
    with pytest.raises(mor.MorError):
        mor.set_wait_budget(0.0)   # below the 1 ms floor the MMA drain needs
    mor.set_wait_budget(1e-3)
    mor.set_wait_budget(1.0)
