"""The autotuner of the local solves' sparse product (mor_autotune).

The first product of each (precision, column count, slot width) is timed in four
launch configurations and the fastest is kept.  Every configuration sums the same
products in the same order, so the bases do not depend on the choice: a build with the
tuner on and one with it off (the first configuration) agree to the run-to-run level
of the mixed path, whose binary32 restriction sums of the coarse level use atomics in
an order that varies from run to run (about 1e-9 in the singular values).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_autotuner_picks_a_configuration_and_keeps_the_results():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2404_06260_gb300 import _build
    _build.build()
    from paper_2404_06260_gb300 import mor
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    opts = mor.basis_opts(rank=p["rank"], oversample=p["oversample"], seed=p["seed"],
                          precision="mixed", cg_rtol=1e-9)
    res = {}
    try:
        for on in (True, False):
            mor.autotune(None)
            mor.autotune(on)
            b = mor.Bases(sd, opts)
            x, info = mor.Reduced(sd, b).solve(rtol=1e-13)
            rep = mor.autotune_report()
            if on:
                # one entry per distinct (precision, column count, slot width) met
                assert len(rep) >= 1
                for e in rep:
                    assert not e["binary64"] and e["columns"] % 4 == 0
                    assert all(t > 0 for t in e["us"])
            else:
                assert rep == []
            res[on] = (b.sigma(), info["energy"])
    finally:
        mor.autotune(None)
        mor.autotune(True)
    s1, e1 = res[True]
    s0, e0 = res[False]
    assert np.max(np.abs(s1 - s0)) <= 1e-7 * s0.max()
    assert abs(e1 - e0) <= 1e-8 * e0
