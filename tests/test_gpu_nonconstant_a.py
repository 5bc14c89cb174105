"""GPU path on the paper's nonconstant-coefficient test (Sec. 7.3), tolerance mode.

a(x) = 10^k sin(100 x) + 10^k + 1 (k = 1, 2, 3; contrast up to 2001 : 1) on a 24^3 Kuhn
cube with 30 seeded k-means subdomains, 6 hops, eps = 1e-2 (Eq. (15)), f = 1, bases from
the randomized sketch with k_i = 64 + 10 columns.

- Parity (binary64 path, k = 3, both H1 forms): the reduced energy b~^T x and the lifted
  solution match the oracle's randomized pipeline (same Philox draws) to 1e-9 / 1e-8.
  Every subdomain keeps the same number of directions, except where an oracle sigma_j
  lies within 1e-6 of eps (a rounding tie).
- With the unweighted H1 form of Sec. 4 this batch has a 7.8e-2 relative reduction error
  at k = 3, the same in the oracle with explicit SVDs.  The local bound is in the
  unweighted norm, while the energy norm weights gradients by up to 2001.  Weighting the
  H1 form by a (h1_weighted) brings it back to 7e-4, the level of k = 1 and 2.
- Trend (weighted form, binary64 and mixed): the relative reduction error against the
  oracle's FE solution does not depend on k (within 15%), and the absolute energy-norm
  error falls by 2.5..3.8 per step of k, as the paper's printed errors do (3.25, 3.17).
"""
import numpy as np
import pytest
from scipy.sparse.linalg import splu

import synth
from oracle import fem, pipeline, reduced

pytestmark = pytest.mark.gpu

EPS = 1e-2


@pytest.fixture(scope="module")
def mor():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2404_06260_gb300 import _build
    _build.build()
    from paper_2404_06260_gb300 import mor as m
    return m


@pytest.fixture(scope="module")
def setup():
    mesh = synth.kuhn_cube(24)
    owner = synth.kmeans_owner(mesh, 30, 1005)
    return mesh, owner


def _gpu(mor, mesh, owner, a, precision, rtol, weighted):
    gm = mor.Mesh(mesh.xyz, mesh.tets, a, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, 6)
    b = mor.Bases(sd, mor.basis_opts(rank=64, oversample=10, seed=1005, precision=precision,
                                     cg_rtol=rtol, eps=EPS, h1_weighted=int(weighted)))
    assert b.converged
    r = mor.Reduced(sd, b)
    x, info = r.solve(rtol=1e-13)
    assert info["converged"]
    return b, info, mor.lift(sd, b, x).cpu().numpy()


def _fe(mesh, a):
    A, bvec, _, free = fem.global_system(mesh, a)
    u = np.zeros(mesh.n_nodes)
    u[free] = splu(A.tocsc()).solve(bvec)
    return u


@pytest.mark.parametrize("weighted", [False, True])
def test_tolerance_mode_parity_at_highest_contrast(mor, setup, weighted):
    mesh, owner = setup
    a = synth.sine_kappa(mesh, 3)
    ref = pipeline.run(mesh, a, owner, 64, 10, 6, 1005, eps=EPS, fe_solution=False,
                       h1_weighted=weighted)
    b, info, u = _gpu(mor, mesh, owner, a, "fp64", 1e-12, weighted)
    assert abs(info["energy"] - ref["E"]) <= 1e-9 * ref["E"]
    for i, ob in enumerate(ref["bases"]):
        tie = np.any(np.abs(ob["sigma"] - EPS) < 1e-6 * EPS)
        assert tie or b.kept[i] == ob["n_kept"], (i, b.kept[i], ob["n_kept"])
    assert reduced.energy_norm(mesh, a, u - ref["u_red"]) <= \
        1e-8 * reduced.energy_norm(mesh, a, ref["u_red"])


def test_weighted_h1_form_restores_the_error_level_at_high_contrast(mor, setup):
    mesh, owner = setup
    a = synth.sine_kappa(mesh, 3)
    u = _fe(mesh, a)
    nu = reduced.energy_norm(mesh, a, u)
    rel = {}
    for weighted in (False, True):
        _, _, ut = _gpu(mor, mesh, owner, a, "fp64", 1e-12, weighted)
        rel[weighted] = reduced.energy_norm(mesh, a, u - ut) / nu
    assert rel[False] > 1e-2
    assert rel[True] < 1e-3


@pytest.mark.parametrize("precision,rtol", [("fp64", 1e-12), ("mixed", 1e-11)])
def test_reduction_error_trend_matches_the_paper(mor, setup, precision, rtol):
    mesh, owner = setup
    rel, absolute = [], []
    for k in (1, 2, 3):
        a = synth.sine_kappa(mesh, k)
        u = _fe(mesh, a)
        _, _, ut = _gpu(mor, mesh, owner, a, precision, rtol, True)
        e = reduced.energy_norm(mesh, a, u - ut)
        absolute.append(e)
        rel.append(e / reduced.energy_norm(mesh, a, u))
    assert max(rel) < 1.15 * min(rel), rel
    assert max(rel) < 1e-3
    for j in (0, 1):
        assert 2.5 < absolute[j] / absolute[j + 1] < 3.8, absolute
