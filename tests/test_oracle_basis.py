"""Pins for the oracle's local basis (Sec. 4, Sec. 5.1, Sec. 6 randomized NLA, App. B)."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.sparse.linalg import splu

import synth
from oracle import basis, fem, subdomains


@pytest.fixture(scope="module")
def cube16():
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    subs = subdomains.all_subdomains(mesh, owner, p["r_hops"])
    return mesh, kappa, owner, p, subs


def test_lemma41_cholesky_block_equals_schur_factor(cube16):
    mesh, kappa, owner, p, subs = cube16
    loc = basis.local_system(mesh, kappa, subs[0])
    R1 = basis.rbb_cholesky(loc["H_plus"], loc["nI"])
    R2 = basis.rbb_schur(loc["H_plus"], loc["nI"])
    assert np.max(np.abs(R1 - R2)) < 1e-12 * np.max(np.abs(R1))
    assert np.allclose(np.tril(R1, -1), 0)


def test_lemma42_trace_norm_is_min_extension_norm(cube16):
    mesh, kappa, owner, p, subs = cube16
    loc = basis.local_system(mesh, kappa, subs[3])
    nI = loc["nI"]
    H = loc["H_plus"].tocsr()
    R_BB = basis.weight_rbb(H, nI)
    beta = np.random.default_rng(0).standard_normal((loc["nB"], 4))
    vI = -splu(H[:nI, :nI].tocsc()).solve(H[:nI, nI:] @ beta)
    v = np.vstack([vI, beta])
    ext = np.einsum("ij,ij->j", v, H @ v)
    assert np.allclose(ext, np.sum((R_BB @ beta) ** 2, axis=0), rtol=1e-11)


def test_local_solution_splits_into_load_part_and_lifting(cube16):
    # Sec. 5.1: u|omega_i = u_{i,0}|omega_i + Z_i (u|boundary), with the lifting of
    # Prob. "aux2" (Eq. (8)) solving A_II u_I = -A_IB z (the paper's matrix Z_i drops that sign)
    mesh, kappa, owner, p, subs = cube16
    A, b, fmap, free = fem.global_system(mesh, kappa)
    u = np.zeros(mesh.n_nodes)
    u[free] = splu(A.tocsc()).solve(b)
    for s in (subs[0], subs[6]):
        loc = basis.local_system(mesh, kappa, s)
        luA = splu(loc["A_II"])
        u0 = luA.solve(loc["b_I"])
        zB = u[s["B"]]
        rec = loc["C"] @ (u0 - luA.solve(loc["A_IB"] @ zB))
        assert np.max(np.abs(rec - u[s["omega"]])) < 1e-12 * np.max(np.abs(u))


def test_weighted_norm_equals_operator_norm(cube16):
    # Eq. (13): ||Z|| = sup ||Z beta||_{1,omega} / ||beta||_trace = ||R_i Z R_BB^{-1}||_2;
    # the sup is the top generalized eigenvalue of (Z^T H_i Z, S_B), S_B = Schur of H^+
    mesh, kappa, owner, p, subs = cube16
    s = subs[1]
    b = basis.local_basis(mesh, kappa, s, rank=4, explicit=True)
    loc = basis.local_system(mesh, kappa, s)
    nI = loc["nI"]
    H = loc["H_plus"].tocsr()
    S_B = H[nI:, nI:].toarray() - H[nI:, :nI] @ splu(H[:nI, :nI].tocsc()).solve(
        H[:nI, nI:].toarray())
    Z = loc["C"] @ splu(loc["A_II"]).solve(loc["A_IB"].toarray())
    N = Z.T @ (loc["H_i"] @ Z)
    w = sla.eigh(0.5 * (N + N.T), 0.5 * (S_B + S_B.T), eigvals_only=True)
    top = np.sqrt(np.sort(w)[::-1][:5])
    assert np.allclose(top, b["sigma"][:5], rtol=1e-9)


def test_randomized_with_full_sketch_equals_explicit_svd(cube16):
    # with k >= M the sketch spans the whole range: the randomized SVD of Eq. (24)
    # gives the singular values and top subspace of the explicit SVD (Eq. (14))
    mesh, kappa, owner, p, subs = cube16
    s = subs[2]
    M = len(s["B"])
    e = basis.local_basis(mesh, kappa, s, rank=10, explicit=True)
    for mode in ("field", "paper"):
        r = basis.local_basis(mesh, kappa, s, rank=10, oversample=M + 5 - 10, seed=3,
                              sketch=mode)
        n = min(len(e["sigma"]), len(r["sigma"]))
        big = e["sigma"][:n] > 1e-8 * e["sigma"][0]
        assert np.allclose(r["sigma"][:n][big], e["sigma"][:n][big], rtol=1e-7,
                           atol=1e-12 * e["sigma"][0])
        assert np.max(np.abs(r["sigma"][:20] - e["sigma"][:20])) < 1e-10 * e["sigma"][0]
        # same top-10 space in the H_i metric: principal angles via H_i-orthonormal cols
        Hi = basis.local_system(mesh, kappa, s)["H_i"]
        G = e["cols"].T @ (Hi @ r["cols"])
        cosines = np.linalg.svd(G, compute_uv=False)
        assert np.min(cosines) > 1 - 1e-10


def test_basis_columns_are_h1_orthonormal(cube16):
    mesh, kappa, owner, p, subs = cube16
    b = basis.local_basis(mesh, kappa, subs[4], rank=8, oversample=5, seed=1)
    Hi = basis.local_system(mesh, kappa, subs[4])["H_i"]
    assert np.allclose(b["cols"].T @ (Hi @ b["cols"]), np.eye(8), atol=1e-10)
    # the diagonal-block update makes Q_i^T A_ii Q_i = I
    assert np.allclose(b["Kii"], np.eye(b["n_kept"]), atol=1e-10)


def test_randomized_singular_values_interlace_explicit(cube16):
    # singular values of Qh^T Y never exceed those of Y (projection)
    mesh, kappa, owner, p, subs = cube16
    s = subs[5]
    e = basis.local_basis(mesh, kappa, s, rank=8, explicit=True)
    r = basis.local_basis(mesh, kappa, s, rank=8, oversample=5, seed=9)
    k = len(r["sigma"])
    assert np.all(r["sigma"] <= e["sigma"][:k] * (1 + 1e-10))
    assert r["sigma"][0] > 0.9 * e["sigma"][0]


def test_range_finder_within_halko_tail_bound(cube16):
    # App. B, Lemma B.2 (Halko et al. Thm 10.8) with t = 2, u = 5: failure
    # probability 2 t^-p + e^{-u^2/2} < 3e-3 for p = 10
    mesh, kappa, owner, p, subs = cube16
    s = subs[7]
    kt, ov = 8, 10
    loc = basis.local_system(mesh, kappa, s)
    luA = splu(loc["A_II"])
    R_i = np.linalg.cholesky(loc["H_i"].toarray()).T
    R_BB = basis.weight_rbb(loc["H_plus"], loc["nI"])
    Z = loc["C"] @ luA.solve(loc["A_IB"].toarray())
    Yf = R_i @ sla.solve_triangular(R_BB, Z.T, trans="T").T
    sig = np.linalg.svd(Yf, compute_uv=False)
    for mode in ("paper", "field"):
        W = basis.sketch_W(mesh, s, loc, kt + ov, 77, mode, R_BB)
        Qh, _ = np.linalg.qr(R_i @ (loc["C"] @ luA.solve(loc["A_IB"] @ W)))
        err = np.linalg.norm(Yf - Qh @ (Qh.T @ Yf), 2)
        t, u = 2.0, 5.0
        c = math.e * math.sqrt(kt + ov) / (ov + 1)
        tail = math.sqrt(np.sum(sig[kt:] ** 2))
        bound = (1 + t * math.sqrt(3 * kt / (ov + 1))) * sig[kt] + t * c * tail + u * t * c * sig[kt]
        assert err <= bound
        assert err >= sig[kt + ov] * (1 - 1e-10)       # no rank-(k+p) space beats the SVD


def test_lemma51_local_bound_in_tolerance_mode(cube16):
    # Lemma 5.1: ||u - v~_i||_{1,omega_i} / ||u||_{1,omega_i^+} < eps with
    # v~_i = u_{i,0} + Z~_i u|B and Z~_i the truncated weighted SVD (Eq. (15))
    mesh, kappa, owner, p, subs = cube16
    A, b, fmap, free = fem.global_system(mesh, kappa)
    u = np.zeros(mesh.n_nodes)
    u[free] = splu(A.tocsc()).solve(b)
    for eps in (1e-1, 3e-2):
        for s in (subs[0], subs[7]):
            loc = basis.local_system(mesh, kappa, s)
            luA = splu(loc["A_II"])
            u0 = loc["C"] @ luA.solve(loc["b_I"])
            R_i = np.linalg.cholesky(loc["H_i"].toarray()).T
            R_BB = basis.weight_rbb(loc["H_plus"], loc["nI"])
            Z = -(loc["C"] @ luA.solve(loc["A_IB"].toarray()))
            Yf = R_i @ sla.solve_triangular(R_BB, Z.T, trans="T").T
            U, sg, Vt = np.linalg.svd(Yf, full_matrices=False)
            m = int(np.sum(sg > eps))
            T = (U[:, :m] * sg[:m]) @ Vt[:m]
            Zt = sla.solve_triangular(R_i, T @ R_BB)
            zB = u[s["B"]]
            d = u[s["omega"]] - (u0 + Zt @ zB)
            num = math.sqrt(d @ (loc["H_i"] @ d))
            up = np.concatenate([u[s["I"]], u[s["B"]]])
            den = math.sqrt(up @ (loc["H_plus"] @ up))
            assert num / den < eps
            # and the bound is attained only through the operator norm: it is loose
            assert num / den < 0.5 * eps


@pytest.mark.parametrize("h1_weighted", [False, True])
def test_field_and_paper_sketch_have_covariance_SB_inverse(h1_weighted):
    # both sketch sources draw W with covariance S_B^{-1} = (R_BB^T R_BB)^{-1}, for the
    # H1 form of Sec. 4 and for its coefficient-weighted variant (the element factors
    # of the field sketch follow the form)
    mesh = synth.kuhn_cube(4)
    kappa = synth.lognormal_kappa(mesh.n_tets, 3)
    owner = synth.slab_owner(4, 2)
    s = subdomains.subdomain_sets(mesh, owner, 0, 1)
    loc = basis.local_system(mesh, kappa, s, h1_weighted=h1_weighted)
    R_BB = basis.weight_rbb(loc["H_plus"], loc["nI"])
    Rinv = sla.solve_triangular(R_BB, np.eye(R_BB.shape[0]))
    cov = Rinv @ Rinv.T
    ncol = 80000
    # E||emp - cov||_F^2 = (||cov||_F^2 + tr(cov)^2) / ncol for Gaussian columns
    sd = math.sqrt((np.sum(cov ** 2) + np.trace(cov) ** 2) / ncol) / np.linalg.norm(cov)
    H = loc["H_plus"].toarray()
    nI = loc["nI"]
    wrong = np.linalg.inv(H[nI:, nI:])          # H_BB^{-1}: ignores the interior
    assert np.linalg.norm(wrong - cov) / np.linalg.norm(cov) > 10 * sd
    for mode in ("paper", "field"):
        W = basis.sketch_W(mesh, s, loc, ncol, 5, mode, R_BB)
        emp = W @ W.T / ncol
        rel = np.linalg.norm(emp - cov) / np.linalg.norm(cov)
        assert rel < 4.0 * sd


def test_weighted_h1_form_reduces_to_the_paper_form_for_unit_coefficient():
    # with k = 1 the coefficient-weighted H1 form is the form of Sec. 4, so the two
    # variants give the same basis
    mesh, _, owner, p = synth.workload("cube16_p2")
    ones = np.ones(mesh.n_tets)
    s = subdomains.subdomain_sets(mesh, owner, 3, p["r_hops"])
    a = basis.local_basis(mesh, ones, s, p["rank"], p["oversample"], p["seed"])
    b = basis.local_basis(mesh, ones, s, p["rank"], p["oversample"], p["seed"],
                          h1_weighted=True)
    assert np.array_equal(a["sigma"], b["sigma"])
    assert np.array_equal(a["Q"], b["Q"])
    kappa = synth.lognormal_kappa(mesh.n_tets, 3)
    c = basis.local_basis(mesh, kappa, s, p["rank"], p["oversample"], p["seed"])
    d = basis.local_basis(mesh, kappa, s, p["rank"], p["oversample"], p["seed"],
                          h1_weighted=True)
    assert not np.allclose(c["sigma"], d["sigma"])   # the variant is not a no-op


def test_gram_form_of_the_weighted_svd_equals_the_printed_form(cube16):
    # Eq. (24) as printed (SVD of B = Qh^T R_i Z R_BB^{-1} with R_BB from the Cholesky
    # factor of H^+) and the Gram form B B^T = T^T S_B^{-1} T (Lemma 4.1: S_B = R_BB^T
    # R_BB, and S_B^{-1} is the B block of (H^+)^{-1}) give the same singular values
    # and the same basis; large subdomains use the Gram form in the oracle
    mesh, kappa, owner, p, subs = cube16
    for i in (0, 6):
        a = basis.local_basis(mesh, kappa, subs[i], 8, 5, 11, rbb="always")
        b = basis.local_basis(mesh, kappa, subs[i], 8, 5, 11, rbb="never")
        assert b["R_BB"] is None and a["R_BB"] is not None
        assert np.max(np.abs(a["sigma"] - b["sigma"])) <= 1e-12 * a["sigma"][0]
        A = a["A_PP"]
        R = b["Q"] - a["Q"] @ (a["Q"].T @ (A @ b["Q"]))
        sin_max = np.sqrt(max(0.0, np.linalg.eigvalsh(R.T @ (A @ R)).max()))
        gap = (a["sigma"][7] - a["sigma"][8]) / a["sigma"][0]
        assert sin_max <= 1e-11 / min(1.0, gap)
