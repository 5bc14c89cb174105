"""Degenerate cases of the method on the GPU path, against the oracle (binary64 path, the
16^3 cube with its lognormal coefficient).

- The smallest sketch, k = 1 (rank 1, no oversampling): one Gaussian column per
  subdomain, so sigma_1 is a single randomized sample; it and the reduced energy match
  the oracle's (the same Philox draws).  Columns 1..3 of every 4-wide block are padding.
- Tolerance mode at its extremes (Eq. (15)): eps above every sigma keeps only the load
  column u_0 of each subdomain; eps far below keeps every sketched direction.
- The smallest partition, two subdomains sharing one interface.
- The widest sketch of the small dense kernels, k = 79 (kp = 80 columns, the limit of
  the shared-memory eigensolver); the narrowest sketch of the wide kernels, k = 80
  (global-memory Jacobi, tiled Grams and row products); and the errors beyond the
  limits (k <= 511 sketch columns, at most 128 basis columns per subdomain).
- The mixed path at k = 1 (three of the four binary32 columns of a pack are padding)
  and at k = 79, within 1e-6 in energy of the binary64 path.

Tolerances as in the 16^3 parity tests: sigma to 1e-10 sigma_1, reduced energy and the
lifted solution to 1e-10 relative.
"""
import numpy as np
import pytest

import synth
from oracle import pipeline, reduced

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
def cube16():
    return synth.workload("cube16_p2")


def _gpu(mor, mesh, kappa, owner, r_hops, rank, oversample, seed, eps=0.0,
         precision="fp64"):
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, r_hops)
    rtol = 1e-13 if precision == "fp64" else 1e-9
    b = mor.Bases(sd, mor.basis_opts(rank=rank, oversample=oversample, seed=seed,
                                     precision=precision, cg_rtol=rtol, eps=eps))
    assert b.converged
    r = mor.Reduced(sd, b)
    x, info = r.solve(rtol=1e-14)
    assert info["converged"]
    return b, info, mor.lift(sd, b, x).cpu().numpy()


def _same_solution(mesh, kappa, ref, info, u):
    assert abs(info["energy"] - ref["E"]) <= 1e-10 * ref["E"]
    assert reduced.energy_norm(mesh, kappa, u - ref["u_red"]) <= \
        1e-10 * reduced.energy_norm(mesh, kappa, ref["u_red"])


def test_smallest_sketch_one_column(mor, cube16):
    mesh, kappa, owner, p = cube16
    ref = pipeline.run(mesh, kappa, owner, 1, 0, p["r_hops"], p["seed"], fe_solution=False)
    b, info, u = _gpu(mor, mesh, kappa, owner, p["r_hops"], 1, 0, p["seed"])
    sg = b.sigma()
    for i, ob in enumerate(ref["bases"]):
        assert abs(sg[i, 0] - ob["sigma"][0]) <= 1e-10 * ob["sigma"][0]
        assert b.kept[i] == ob["n_kept"] == 2          # u_0 and the one direction
    _same_solution(mesh, kappa, ref, info, u)
    _mixed_close(mor, mesh, kappa, owner, p, 1, 0, b, u)


def _mixed_close(mor, mesh, kappa, owner, p, rank, oversample, b64, u64):
    bm, _, um = _gpu(mor, mesh, kappa, owner, p["r_hops"], rank, oversample, p["seed"],
                     precision="mixed")
    assert np.array_equal(bm.kept, b64.kept)
    assert reduced.energy_norm(mesh, kappa, um - u64) <= \
        1e-6 * reduced.energy_norm(mesh, kappa, u64)


@pytest.mark.parametrize("which", ["above_all", "below_all"])
def test_tolerance_mode_extremes(mor, cube16, which):
    mesh, kappa, owner, p = cube16
    k = p["rank"] + p["oversample"]
    ref0 = pipeline.run(mesh, kappa, owner, p["rank"], p["oversample"], p["r_hops"],
                        p["seed"], fe_solution=False)
    sig = np.concatenate([ob["sigma"][:k] for ob in ref0["bases"]])
    assert sig.min() > 1e-8
    eps = 10.0 * sig.max() if which == "above_all" else 1e-12
    ref = pipeline.run(mesh, kappa, owner, p["rank"], p["oversample"], p["r_hops"],
                       p["seed"], eps=eps, fe_solution=False)
    b, info, u = _gpu(mor, mesh, kappa, owner, p["r_hops"], p["rank"], p["oversample"],
                      p["seed"], eps=eps)
    m_or = np.array([ob["m"] for ob in ref["bases"]])
    assert np.all(m_or == (0 if which == "above_all" else k))
    assert np.array_equal(b.kept, [ob["n_kept"] for ob in ref["bases"]])
    if which == "above_all":
        assert np.all(b.kept == 1)                     # u_0 alone
    _same_solution(mesh, kappa, ref, info, u)


def test_two_subdomains(mor, cube16):
    mesh, kappa, owner, p = cube16
    two = (mesh.xyz[:, 0] > 0.5).astype(owner.dtype)
    ref = pipeline.run(mesh, kappa, two, p["rank"], p["oversample"], p["r_hops"], p["seed"],
                       fe_solution=False)
    b, info, u = _gpu(mor, mesh, kappa, two, p["r_hops"], p["rank"], p["oversample"],
                      p["seed"])
    sg = b.sigma()
    k = p["rank"] + p["oversample"]
    for i, ob in enumerate(ref["bases"]):
        assert np.max(np.abs(sg[i, :k] - ob["sigma"][:k])) <= 1e-10 * ob["sigma"][0]
    _same_solution(mesh, kappa, ref, info, u)


def test_widest_sketch_79_columns(mor, cube16):
    mesh, kappa, owner, p = cube16
    rank, over = 69, 10
    ref = pipeline.run(mesh, kappa, owner, rank, over, p["r_hops"], p["seed"],
                       fe_solution=False)
    b, info, u = _gpu(mor, mesh, kappa, owner, p["r_hops"], rank, over, p["seed"])
    sg = b.sigma()
    assert sg.shape[1] == 79
    for i, ob in enumerate(ref["bases"]):
        assert np.max(np.abs(sg[i] - ob["sigma"][:79])) <= 1e-10 * ob["sigma"][0]
    assert np.array_equal(b.kept, [ob["n_kept"] for ob in ref["bases"]])
    _same_solution(mesh, kappa, ref, info, u)
    _mixed_close(mor, mesh, kappa, owner, p, rank, over, b, u)


def test_first_wide_sketch_80_columns(mor, cube16):
    mesh, kappa, owner, p = cube16
    rank, over = 70, 10
    ref = pipeline.run(mesh, kappa, owner, rank, over, p["r_hops"], p["seed"],
                       fe_solution=False)
    b, info, u = _gpu(mor, mesh, kappa, owner, p["r_hops"], rank, over, p["seed"])
    sg = b.sigma()
    assert sg.shape[1] == 80
    for i, ob in enumerate(ref["bases"]):
        assert np.max(np.abs(sg[i] - ob["sigma"][:80])) <= 1e-10 * ob["sigma"][0]
    assert np.array_equal(b.kept, [ob["n_kept"] for ob in ref["bases"]])
    _same_solution(mesh, kappa, ref, info, u)


def test_sketch_and_basis_width_limits_are_errors(mor, cube16):
    mesh, kappa, owner, p = cube16
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    with pytest.raises(mor.MorError, match="<= 511"):
        mor.Bases(sd, mor.basis_opts(rank=100, oversample=412, seed=p["seed"], eps=1e-30))
    with pytest.raises(mor.MorError, match="<= 128"):
        mor.Bases(sd, mor.basis_opts(rank=130, oversample=10, seed=p["seed"]))
