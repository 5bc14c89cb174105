"""Pins for the oracle's stitching, projection and reduced solve (Def. 3.1, Eq. (23),
Sec. 6 step 3, Sec. 7.1)."""
import math

import numpy as np
import pytest

import synth
from conftest import golden
from oracle import fem, pipeline, reduced


def _paper_load(x, y, z):
    return 60.0 * ((1 - x) * x * (1 - y) * y + (1 - x) * x * (1 - z) * z +
                   (1 - y) * y * (1 - z) * z)


@pytest.fixture(scope="module")
def cube16_run():
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    out = pipeline.run(mesh, kappa, owner, p["rank"], p["oversample"], p["r_hops"], p["seed"])
    return mesh, kappa, owner, p, out


def test_interface_projection_equals_explicit_qtaq(cube16_run):
    # Sec. 6 step 3: K~ built from step-2 diagonal blocks and A_0 on omega_0 equals
    # Q^T A Q with the assembled global A (Eq. (23))
    mesh, kappa, owner, p, out = cube16_run
    A, b, _, _ = fem.global_system(mesh, kappa)
    K, bt = reduced.project_explicit(A, b, reduced.stitched_Q(mesh, out["bases"]))
    assert np.max(np.abs(K - out["K"])) < 1e-12 * np.max(np.abs(K))
    assert np.allclose(bt, out["bt"], rtol=1e-12, atol=1e-18)


def test_reduced_matrix_is_spd_with_identity_diagonal_blocks(cube16_run):
    mesh, kappa, owner, p, out = cube16_run
    K = out["K"]
    assert np.allclose(K, K.T)
    assert np.linalg.eigvalsh(K).min() > 0
    off = reduced.offsets(out["bases"])
    for i in range(len(out["bases"])):
        blk = K[off[i]:off[i + 1], off[i]:off[i + 1]]
        assert np.allclose(blk, np.eye(blk.shape[0]), atol=1e-10)
    # only neighbour pairs couple; 2x2x2 boxes couple every pair
    assert len(out["pairs"]) > 0


def test_galerkin_energy_below_fe_energy_and_monotone_in_rank():
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    k = 14
    E = []
    for m in (2, 6, 12):
        o = pipeline.run(mesh, kappa, owner, m, k - m, p["r_hops"], p["seed"])
        E.append(o["E"])
        E_fe = o["E_fe"]
    assert E[0] < E[1] < E[2] <= E_fe * (1 + 1e-13)


@pytest.mark.parametrize("explicit,h1_weighted", [(True, False), (False, False),
                                                  (False, True)])
def test_full_rank_basis_reproduces_fe_solution(explicit, h1_weighted):
    # Eq. (9): {u_{i,0}, Z_i phi_1..M} represents the local solution for any trace, so
    # stitching the full bases reproduces the FE solution (Sec. 5.2 splitting); the
    # inner product only weights the SVD, so this holds for the weighted variant too
    n = 12
    mesh = synth.kuhn_cube(n)
    kappa = synth.lognormal_kappa(mesh.n_tets, 7)
    owner = synth.slab_owner(n, 2)
    out = pipeline.run(mesh, kappa, owner, rank=130, oversample=0, r_hops=2, seed=1,
                       explicit=explicit, keep_all=True, tau=1e-15, h1_weighted=h1_weighted)
    for b, s in zip(out["bases"], out["subs"]):
        assert b["n_kept"] < len(s["owned"])          # a genuine reduction
    assert out["red_err"] < 1e-12


def test_reduced_method_tracks_fe_error_at_paper_tolerance():
    # Sec. 7.1 / Table 1: at eps = 1e-2 the reduction error is O(1e-4) and far below
    # the FE error, so u~ converges like u (first order in h)
    errs_fe, errs_red = [], []
    for n, parts, r in ((8, 2, 2), (16, 2, 4)):
        mesh = synth.kuhn_cube(n)
        owner = synth.box_owner(n, parts)
        out = pipeline.run(mesh, np.ones(mesh.n_tets), owner, rank=0, oversample=0,
                           r_hops=r, seed=1, explicit=True, eps=1e-2, f=_paper_load)
        errs_fe.append(math.sqrt(1 - out["E_fe"]))
        errs_red.append(math.sqrt(1 - out["E"]))
        assert out["red_err"] < 1e-3
        assert abs(errs_red[-1] - errs_fe[-1]) < 1e-3 * errs_fe[-1]
    assert 0.9 < math.log2(errs_red[0] / errs_red[1]) < 1.1
    # the paper's reduction errors at eps = 1e-2 (Table 1, cases 4-7) are 9e-5..2.6e-4
    assert out["red_err"] < 10 * max(2.6e-4, 9.0e-5)


def test_stitching_partitions_any_nodal_function():
    # Def. 3.1 with owned interiors: sum_i S_i(v|omega_i) = v for every v (Sec. 5.2)
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    from oracle.subdomains import all_subdomains
    subs = all_subdomains(mesh, owner, p["r_hops"])
    v = np.random.default_rng(1).standard_normal(mesh.n_nodes) * (mesh.dirichlet == 0)
    acc = np.zeros(mesh.n_nodes)
    for s in subs:
        w = np.zeros(mesh.n_nodes)
        w[s["omega"]] = v[s["omega"]]       # v restricted to omega_i
        sw = np.zeros(mesh.n_nodes)
        sw[s["owned"]] = w[s["owned"]]      # S_i: keep interior nodes, zero elsewhere
        acc += sw
    assert np.array_equal(acc, v)
