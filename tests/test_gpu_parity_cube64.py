"""GPU path vs the oracle at the benchmarked size (64^3 cube, 64 subdomains, rank 32 + 10,
lognormal coefficient), in the launch configuration bench.py times (MOR_MIXED,
cg_rtol 1e-9) and in binary64.

The oracle computes sampled outputs one subdomain at a time: subdomain 0, the corner
box (|I| = 12,167), takes about 15 s on the CPU, and subdomain 21, an interior box
with the largest extension (|I| = 27,080, the subdomain with the most coarse-level
aggregates), about 40 s.  Sampled outputs: singular values, subspaces and the
rotation-invariant projected load Q_i b~_i of subdomains 0 and 21, and the
rotation-invariant interface blocks Q_i K~_ij Q_j^T of the neighbour pairs (0, 1) and
(21, 22).  Every subdomain's index sets and the sketch right-hand side of sampled
subdomains are checked too.  Properties that hold at any size are checked on the whole
batch: K~ symmetric positive definite with identity diagonal blocks, Q_i^T A_ii Q_i = I,
the reduced solution against a dense solve of the same K~, and the mixed-precision
reduced solution within 1e-6 relative energy of the binary64 one.

Tolerances: binary64 with cg_rtol 1e-11 perturbs the Gram G_B by ~1e-11 ||G_B||, so
|ds| <= 1e-9 s_1 leaves two orders of margin; the subspace bound is that over the gap
(Davis-Kahan).  The mixed path solves to 1e-9 in binary64-measured residuals, so its
singular values are checked to 1e-7 s_1.
"""
import numpy as np
import pytest

import synth
from oracle import basis as obasis
from oracle import fem as ofem
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
def cube64(mor):
    mesh, kappa, owner, p = synth.workload("cube64_p4")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    return mesh, kappa, owner, p, sd


SAMPLED = (0, 1, 21, 22)


@pytest.fixture(scope="module")
def oracle64(cube64):
    mesh, kappa, owner, p, sd = cube64
    adj = osub.node_adjacency(mesh.tets, mesh.n_nodes)
    out = {}
    for i in SAMPLED:
        s = osub.subdomain_sets(mesh, owner, i, p["r_hops"], adj)
        out[i] = obasis.local_basis(mesh, kappa, s, p["rank"], p["oversample"], p["seed"])
    return out


@pytest.fixture(scope="module")
def oracle_sub0(oracle64):
    return oracle64[0]


@pytest.fixture(scope="module")
def gpu64(mor, cube64):
    mesh, kappa, owner, p, sd = cube64
    out = {}
    for prec, rt in (("fp64", 1e-11), ("mixed", 1e-9)):
        opts = mor.basis_opts(rank=p["rank"], oversample=p["oversample"], seed=p["seed"],
                              precision=prec, cg_rtol=rt)
        b = mor.Bases(sd, opts)
        assert b.converged, prec
        r = mor.Reduced(sd, b)
        x, info = r.solve(rtol=1e-12)
        assert info["converged"], prec
        out[prec] = (b, r, x, info, mor.lift(sd, b, x))
    return out


def test_index_sets_bit_exact_for_every_subdomain(cube64):
    mesh, kappa, owner, p, sd = cube64
    adj = osub.node_adjacency(mesh.tets, mesh.n_nodes)
    assert sd.n_sub == 64
    for i in range(sd.n_sub):
        s = osub.subdomain_sets(mesh, owner, i, p["r_hops"], adj)
        for which, key in enumerate(["I", "B", "omega", "owned", "plus_tets", "omega_tets"]):
            assert np.array_equal(sd.indices(i, which), s[key]), (i, key)


def test_sketch_rhs_sampled(mor, cube64):
    mesh, kappa, owner, p, sd = cube64
    k = p["rank"] + p["oversample"]
    opts = mor.basis_opts(rank=p["rank"], oversample=p["oversample"], seed=p["seed"],
                          precision="fp64")
    for i in (0, 21, 63):
        s = osub.subdomain_sets(mesh, owner, i, p["r_hops"])
        loc = obasis.local_system(mesh, kappa, s)
        ref = obasis.field_sketch_rhs(mesh, s, loc, k, p["seed"])
        got = mor.sketch_rhs(sd, opts, i)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref)), i


def _gap(sig, m):
    return (sig[m - 1] - sig[m]) / sig[0]


@pytest.mark.parametrize("sub", [0, 21])
def test_sampled_singular_values_and_subspace(cube64, oracle64, gpu64, sub):
    mesh, kappa, owner, p, sd = cube64
    ob = oracle64[sub]
    if sub == 21:   # the interior box: the largest extension of the batch
        assert sd.counts[sub, 0] == sd.counts[:, 0].max() == 27080
    ref = ob["sigma"]
    m = p["rank"]
    gap = _gap(ref, m)
    for prec, tol in (("fp64", 1e-9), ("mixed", 1e-7)):
        b = gpu64[prec][0]
        sig = b.sigma()[sub]
        n = min(len(ref), len(sig))
        assert np.max(np.abs(sig[:n] - ref[:n])) <= tol * ref[0], prec
        A = ob["A_PP"]
        Qg = b.Q(sub)[:, :b.kept[sub]]
        Qo = ob["Q"]
        assert Qg.shape[1] == Qo.shape[1]
        R = Qg - Qo @ (Qo.T @ (A @ Qg))
        sin_max = np.sqrt(max(0.0, np.linalg.eigvalsh(R.T @ (A @ R)).max()))
        assert sin_max <= tol / min(1.0, gap), (prec, sin_max, gap)
        # Q_i b~_i = Q_i Q_i^T b_P does not depend on the rotation of Q_i
        got = Qg @ b.bt()[sub, :b.kept[sub]]
        want = Qo @ ob["bt"]
        assert np.max(np.abs(got - want)) <= tol / min(1.0, gap) * np.max(np.abs(want)), prec


@pytest.mark.parametrize("pair", [(0, 1), (21, 22)])
def test_sampled_interface_blocks(cube64, oracle64, gpu64, pair):
    # Eq. (23): K~_ij = Q_i^T A_0[P_i, P_j] Q_j, compared in the rotation-invariant form
    # Q_i K~_ij Q_j^T on the interface rows and columns (the owned nodes of i and j
    # coupled by A_0).  A_0[P_i, P_j] comes from the elements with vertices in both
    # P_i and P_j, all of which lie in omega_0.
    mesh, kappa, owner, p, sd = cube64
    i, j = pair
    oi, oj = oracle64[i], oracle64[j]
    ow = owner[mesh.tets]
    t = np.flatnonzero(np.any(ow == i, axis=1) & np.any(ow == j, axis=1))
    G, vol = ofem.tet_geometry(mesh.xyz, mesh.tets[t])
    fmap, free = ofem.free_map(mesh.dirichlet)
    A0 = ofem.assemble_matrix(mesh.tets[t], ofem.stiffness_elements(G, vol, kappa[t]), fmap,
                              len(free)).tocsr()
    Aij = A0[fmap[oi["owned"]]][:, fmap[oj["owned"]]].toarray()
    gi = np.flatnonzero(np.any(Aij != 0, axis=1))
    gj = np.flatnonzero(np.any(Aij != 0, axis=0))
    assert len(gi) > 0 and len(gj) > 0
    ref = (oi["Q"][gi] @ (oi["Q"].T @ Aij @ oj["Q"])) @ oj["Q"][gj].T
    gap = min(_gap(oi["sigma"], p["rank"]), _gap(oj["sigma"], p["rank"]))
    for prec, tol in (("fp64", 1e-9), ("mixed", 1e-7)):
        b, r = gpu64[prec][0], gpu64[prec][1]
        K = r.dense()
        kq = b.kq
        ki, kj = b.kept[i], b.kept[j]
        Kg = K[i * kq:i * kq + ki, j * kq:j * kq + kj]
        got = b.Q(i)[gi, :ki] @ Kg @ b.Q(j)[gj, :kj].T
        assert np.max(np.abs(got - ref)) <= tol / min(1.0, gap) * np.max(np.abs(ref)), prec


def test_reduced_solve_matches_dense_solve_at_full_size(gpu64):
    # the batched reduced CG (stopped at a relative residual of 1e-12) against LAPACK's
    # Cholesky solve of the same K~ and b~: the error of x is at most cond(K~) times the
    # residual, and the energy error is second order in it
    import scipy.linalg as sla
    for prec in ("fp64", "mixed"):
        b, r, x, info, u = gpu64[prec]
        K = r.dense()
        bt = b.bt().ravel()
        xd = sla.cho_solve(sla.cho_factor(K), bt)
        xg = x.cpu().numpy()
        ev = np.linalg.eigvalsh(K)
        tol = 10.0 * (ev[-1] / ev[0]) * 1e-12
        assert np.linalg.norm(xg - xd) <= tol * np.linalg.norm(xd), (prec, tol)
        assert abs(info["energy"] - bt @ xd) <= 1e-10 * (bt @ xd), prec


def test_reduced_matrix_properties_at_full_size(gpu64):
    for prec in ("fp64", "mixed"):
        b, r, x, info, u = gpu64[prec]
        K = r.dense()
        kq = b.kq
        assert np.allclose(K, K.T, atol=1e-12)
        for i in range(len(b.kept)):
            blk = K[i * kq:(i + 1) * kq, i * kq:(i + 1) * kq]
            assert np.array_equal(blk, np.eye(kq))
        assert np.linalg.eigvalsh(K).min() > 0


def test_bases_are_energy_orthonormal_at_full_size(mor, cube64, gpu64, oracle_sub0):
    # Q_i^T A_ii Q_i = I is what makes the diagonal blocks the identity; check it on the
    # sampled subdomain with the oracle's A[P_0, P_0]
    b = gpu64["mixed"][0]
    Q = b.Q(0)[:, :b.kept[0]]
    A = oracle_sub0["A_PP"]
    assert np.allclose(Q.T @ (A @ Q), np.eye(Q.shape[1]), atol=1e-8)


def test_mixed_within_1e6_energy_of_fp64_at_full_size(mor, cube64, gpu64):
    mesh, kappa, owner, p, sd = cube64
    u_m, u_d = gpu64["mixed"][4], gpu64["fp64"][4]
    e = mor.energy_norm(sd, u_m, u_d) / mor.energy_norm(sd, u_d)
    assert e <= 1e-6, e
