"""Streamed plans (mor_build_subdomains_streamed): the 64^3 workload built in waves of 10
subdomains (7 waves) against the one-shot plan.

Each wave runs the same per-subdomain arithmetic; only the sweeps of the iterative
solves (which depend on when all subdomains of a launch have converged) differ, so
results agree to the solve tolerance: with cg_rtol 1e-11 in binary64 the singular
values agree to 1e-9 sigma_1, the kept counts exactly, and the reduced energy and lifted
solution to 1e-9 / 1e-8.  The mixed path stays within 1e-6 in energy.
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


@pytest.fixture(scope="module")
def cube64(mor):
    mesh, kappa, owner, p = synth.workload("cube64_p4")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    full = mor.Subdomains(gm, owner, p["r_hops"])
    waves = mor.Subdomains(gm, owner, p["r_hops"], wave=10)
    return p, full, waves


def _run(mor, sd, p, precision, rtol):
    b = mor.Bases(sd, mor.basis_opts(rank=p["rank"], oversample=p["oversample"], seed=p["seed"],
                                     precision=precision, cg_rtol=rtol))
    assert b.converged
    r = mor.Reduced(sd, b)
    x, info = r.solve(rtol=1e-13)
    assert info["converged"]
    return b, info, mor.lift(sd, b, x)


def test_streamed_plan_reports_global_part_only(mor, cube64):
    p, full, waves = cube64
    assert waves.n_sub == full.n_sub == 64
    assert np.array_equal(waves.counts[:, 3], full.counts[:, 3])     # owned DOFs
    assert np.array_equal(waves.counts[:, 6], full.counts[:, 6])     # hops
    assert np.all(waves.counts[:, 0] == -1)
    with pytest.raises(mor.MorError):
        waves.indices(0, 0)


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-11), ("mixed", 1e-9)])
def test_waves_match_the_one_shot_plan(mor, cube64, precision, rtol):
    p, full, waves = cube64
    bf, inf_f, uf = _run(mor, full, p, precision, rtol)
    bw, inf_w, uw = _run(mor, waves, p, precision, rtol)
    assert np.array_equal(bf.kept, bw.kept)
    e = mor.energy_norm(full, uw, uf) / mor.energy_norm(full, uf)
    if precision == "fp64":
        sf, sw = bf.sigma(), bw.sigma()
        assert np.max(np.abs(sf - sw)) <= 1e-9 * np.max(sf)
        assert abs(inf_f["energy"] - inf_w["energy"]) <= 1e-9 * inf_f["energy"]
        assert e <= 1e-8, e
    else:
        assert e <= 1e-6, e
