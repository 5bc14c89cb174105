"""GPU path vs the CPU oracle on the 16^3 cube (8 subdomains, rank 8 + 5, lognormal
coefficient), through the C ABI.

Tolerances (binary64 path; the oracle uses direct solves, the GPU iterative ones):
  - index sets and Philox/Box-Muller normals: bit-exact (integer work; the normals
    are binary32 values produced by a fixed operation sequence);
  - sketch right-hand side L xi: 1e-12 relative (binary64 element Cholesky factors);
  - singular values: |s_gpu - s_oracle| <= 1e-10 s_1 (normwise; a local-solve residual
    of 1e-13 relative perturbs the 13 x 13 Gram G_B by ~1e-13 ||G_B||);
  - bases: principal angles in the A[P_i,P_i] inner product below 1e-10 / gap, with
    gap = (s_m - s_{m+1}) / s_1 (Davis-Kahan: a subspace moves by perturbation / gap);
  - reduced energy and K~ eigenvalues: 1e-10 relative; lifted u~: 1e-10 in the A-norm.
"""
import numpy as np
import pytest

import synth
from oracle import basis as obasis
from oracle import pipeline, reduced
from oracle import subdomains as osub

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
def cube16(mor):
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    return mesh, kappa, owner, p, sd


@pytest.fixture(scope="module")
def oracle16(cube16):
    mesh, kappa, owner, p, sd = cube16
    return pipeline.run(mesh, kappa, owner, p["rank"], p["oversample"], p["r_hops"],
                        p["seed"], fe_solution=False)


@pytest.fixture(scope="module")
def gpu16(mor, cube16):
    mesh, kappa, owner, p, sd = cube16
    opts = mor.basis_opts(rank=p["rank"], oversample=p["oversample"], seed=p["seed"],
                          precision="fp64", cg_rtol=1e-13)
    bases = mor.Bases(sd, opts)
    red = mor.Reduced(sd, bases)
    x, info = red.solve(rtol=1e-14)
    u = mor.lift(sd, bases, x)
    return bases, red, x, info, u


def test_subdomain_sets_bit_exact(cube16):
    mesh, kappa, owner, p, sd = cube16
    assert sd.n_sub == 8
    for i in range(sd.n_sub):
        s = osub.subdomain_sets(mesh, owner, i, p["r_hops"])
        for which, key in enumerate(["I", "B", "omega", "owned", "plus_tets", "omega_tets"]):
            assert np.array_equal(sd.indices(i, which), s[key]), (i, key)


def test_sketch_rhs_matches_oracle(mor, cube16):
    mesh, kappa, owner, p, sd = cube16
    k = p["rank"] + p["oversample"]
    opts = mor.basis_opts(rank=p["rank"], oversample=p["oversample"], seed=p["seed"],
                          precision="fp64")
    for i in (0, 5):
        s = osub.subdomain_sets(mesh, owner, i, p["r_hops"])
        loc = obasis.local_system(mesh, kappa, s)
        ref = obasis.field_sketch_rhs(mesh, s, loc, k, p["seed"])
        got = mor.sketch_rhs(sd, opts, i)
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_singular_values_match_oracle(cube16, oracle16, gpu16):
    bases = gpu16[0]
    sig = bases.sigma()
    for i, b in enumerate(oracle16["bases"]):
        ref = b["sigma"]
        n = min(len(ref), sig.shape[1])
        assert np.max(np.abs(sig[i, :n] - ref[:n])) <= 1e-10 * ref[0], i


def test_bases_span_the_oracle_subspaces(cube16, oracle16, gpu16):
    mesh, kappa, owner, p, sd = cube16
    bases = gpu16[0]
    m = p["rank"]
    for i, b in enumerate(oracle16["bases"]):
        Qg = bases.Q(i)[:, :bases.kept[i]]
        Qo = b["Q"]
        assert Qg.shape[1] == Qo.shape[1]
        A = b["A_PP"]
        assert np.allclose(Qg.T @ (A @ Qg), np.eye(Qg.shape[1]), atol=1e-10)
        # largest principal-angle sine = ||(I - P_o) Q_g|| in the A inner product, with
        # P_o the A-orthogonal projector onto span(Q_o) (accurate for tiny angles)
        R = Qg - Qo @ (Qo.T @ (A @ Qg))
        sin_max = np.sqrt(max(0.0, np.linalg.eigvalsh(R.T @ (A @ R)).max()))
        s = b["sigma"]
        gap = (s[m - 1] - s[m]) / s[0]
        assert sin_max <= 1e-10 / min(1.0, gap), (i, sin_max, gap)


def _gap(sig, m):
    return (sig[m - 1] - sig[m]) / sig[0]


def test_projected_load_matches_oracle(cube16, oracle16, gpu16):
    # b~_i = Q_i^T b_P depends on which A-orthonormal basis Q_i of the local space is
    # chosen, but Q_i b~_i = Q_i Q_i^T b_P does not: two such bases differ by an
    # orthogonal rotation O, and (Q O)(Q O)^T = Q Q^T.  Compare that vector element by
    # element.
    mesh, kappa, owner, p, sd = cube16
    bases = gpu16[0]
    bt = bases.bt()
    for i, b in enumerate(oracle16["bases"]):
        Qg = bases.Q(i)[:, :bases.kept[i]]
        got = Qg @ bt[i, :bases.kept[i]]
        ref = b["Q"] @ b["bt"]
        tol = 1e-10 / min(1.0, _gap(b["sigma"], p["rank"]))
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)), i


def test_interface_blocks_match_oracle_for_every_pair(cube16, oracle16, gpu16):
    # K~_ij = Q_i^T A_0[P_i, P_j] Q_j (Eq. (23)) in the rotation-invariant form
    # Q_i K~_ij Q_j^T = (Q_i Q_i^T) A_0[P_i, P_j] (Q_j Q_j^T), element by element over
    # the owned nodes of both subdomains, for every neighbour pair of the batch
    mesh, kappa, owner, p, sd = cube16
    bases, red = gpu16[0], gpu16[1]
    K = red.dense()
    kq = bases.kq
    off = reduced.offsets(oracle16["bases"])
    Ko = oracle16["K"]
    assert len(oracle16["pairs"]) > 0
    for i, j in oracle16["pairs"]:
        bi, bj = oracle16["bases"][i], oracle16["bases"][j]
        ki, kj = bases.kept[i], bases.kept[j]
        Kg = K[i * kq:i * kq + ki, j * kq:j * kq + kj]
        got = bases.Q(i)[:, :ki] @ Kg @ bases.Q(j)[:, :kj].T
        ref = bi["Q"] @ Ko[off[i]:off[i + 1], off[j]:off[j + 1]] @ bj["Q"].T
        gap = min(_gap(bi["sigma"], p["rank"]), _gap(bj["sigma"], p["rank"]))
        tol = 1e-10 / min(1.0, gap)
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)), (i, j)


def test_reduced_system_and_solution_match_oracle(cube16, oracle16, gpu16):
    mesh, kappa, owner, p, sd = cube16
    bases, red, x, info, u = gpu16
    K = red.dense()
    # drop the identity rows/cols of unused padding columns
    keep = np.concatenate([np.arange(i * bases.kq, i * bases.kq + bases.kept[i])
                           for i in range(sd.n_sub)])
    Kg = K[np.ix_(keep, keep)]
    assert np.allclose(Kg, Kg.T, atol=1e-13)
    ev_g = np.linalg.eigvalsh(Kg)
    ev_o = np.linalg.eigvalsh(oracle16["K"])
    assert ev_g.min() > 0
    assert np.max(np.abs(ev_g - ev_o)) <= 1e-10 * ev_o.max()
    assert info["converged"]
    assert abs(info["energy"] - oracle16["E"]) <= 1e-10 * oracle16["E"]
    ug = u.cpu().numpy()
    err = reduced.energy_norm(mesh, kappa, ug - oracle16["u_red"])
    assert err <= 1e-10 * reduced.energy_norm(mesh, kappa, oracle16["u_red"])


def test_gpu_energy_norm_matches_oracle(mor, cube16, oracle16, gpu16):
    import torch
    mesh, kappa, owner, p, sd = cube16
    u_or = torch.as_tensor(oracle16["u_red"], device="cuda")
    got = mor.energy_norm(sd, u_or)
    assert np.isclose(got, reduced.energy_norm(mesh, kappa, oracle16["u_red"]), rtol=1e-12)


def test_mixed_precision_within_1e6_energy_error(mor, cube16, gpu16):
    mesh, kappa, owner, p, sd = cube16
    u_d = gpu16[4]
    opts = mor.basis_opts(rank=p["rank"], oversample=p["oversample"], seed=p["seed"],
                          precision="mixed", cg_rtol=1e-9)
    bm = mor.Bases(sd, opts)
    assert bm.converged
    rm = mor.Reduced(sd, bm)
    xm, info = rm.solve(rtol=1e-12)
    um = mor.lift(sd, bm, xm)
    e = mor.energy_norm(sd, um, u_d) / mor.energy_norm(sd, u_d)
    assert e <= 1e-6, e


def test_full_rank_basis_reproduces_fe_solution(mor):
    # Eq. (9): with every boundary direction kept, the stitched bases span the FE
    # solution; two slabs of the 8^3 cube, |B| = 49 boundary nodes, rank 49
    import torch
    n = 8
    mesh = synth.kuhn_cube(n)
    kappa = synth.lognormal_kappa(mesh.n_tets, 7)
    owner = synth.slab_owner(n, 2)
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, 2)
    M = int(sd.counts[:, 1].max())
    opts = mor.basis_opts(rank=M, oversample=4, seed=3, precision="fp64", cg_rtol=1e-13,
                          tau=1e-15, orth_tol=1e-28)
    bases = mor.Bases(sd, opts)
    assert np.all(bases.kept < sd.counts[:, 3])
    red = mor.Reduced(sd, bases)
    x, info = red.solve(rtol=1e-14)
    u = mor.lift(sd, bases, x)
    ref = pipeline.run(mesh, kappa, owner, rank=1, oversample=0, r_hops=2, seed=1,
                       explicit=True)
    u_fe = torch.as_tensor(ref["u"], device="cuda")
    err = mor.energy_norm(sd, u, u_fe) / mor.energy_norm(sd, u_fe)
    assert err < 1e-10, err


def test_host_array_entry_point_gives_the_same_bases(mor, cube16, gpu16):
    # mor_build_subdomains_host copies the mesh itself: the same plan (bit-exact index
    # sets) and the same bases; the CG restriction sums use shared-memory atomics, whose
    # order varies from run to run, so the results agree to rounding, not to the bit
    mesh, kappa, owner, p, sd = cube16
    sdh = mor.Subdomains.from_host(mesh.xyz, mesh.tets, kappa, mesh.dirichlet, owner,
                                   p["r_hops"])
    assert np.array_equal(sdh.counts, sd.counts)
    for i in range(sd.n_sub):
        for which in range(6):
            assert np.array_equal(sdh.indices(i, which), sd.indices(i, which))
    opts = mor.basis_opts(rank=p["rank"], oversample=p["oversample"], seed=p["seed"],
                          precision="fp64", cg_rtol=1e-13)
    bh = mor.Bases(sdh, opts)
    b = gpu16[0]
    s0 = b.sigma()
    assert np.max(np.abs(bh.sigma() - s0)) <= 1e-12 * s0.max()
    assert np.array_equal(bh.kept, b.kept)
    for i in range(sd.n_sub):
        Q1, Q0 = bh.Q(i)[:, :b.kept[i]], b.Q(i)[:, :b.kept[i]]
        # the same span: the least-squares projection of one basis onto the other
        P = Q0 @ np.linalg.lstsq(Q0, Q1, rcond=None)[0]
        assert np.max(np.abs(P - Q1)) <= 1e-8 * np.max(np.abs(Q1))
