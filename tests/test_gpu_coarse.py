"""Coarse level of the local preconditioner (M^{-1} = D^{-1} + Z E^{-1} Z^T).

The aggregate matrices E = Z^T A Z are inverted by blocked Gauss-Jordan elimination in
binary32 on the diagonally scaled block W = S E S (S = diag(E)^{-1/2}).  For symmetric
positive definite input that elimination needs no pivoting and is backward stable, so
the computed inverse is within a small multiple of n u kappa(W) of the exact one
(u = 2^-24; the checks allow 10 n u kappa(W) in the 2-norm, relative).  Sizes cover one
pivot, a ragged last pivot block (63, 65, 565) and the 1024 cap.  The preconditioner
changes iteration counts only: finer aggregates (coarse_rows 35, the mixed default, against
100) must cut the iterations of the 64^3 build by at least a tenth and leave its singular
values and reduced energy where the CG tolerance puts them.
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


def _spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.logspace(0, np.log10(cond), n)
    d = 10.0 ** rng.uniform(-3, 3, n)          # a scaling the inversion must undo
    return (d[:, None] * (Q * lam) @ Q.T) * d[None, :]


@pytest.mark.parametrize("n", [1, 7, 63, 64, 65, 200, 565, 1024])
def test_coarse_inverse_within_the_backward_error_bound(mor, n):
    import torch
    E = _spd(n, n)
    X = mor.coarse_inverse(torch.as_tensor(E, device="cuda")).cpu().numpy()
    assert np.array_equal(X, X.T)
    s = 1.0 / np.sqrt(np.diag(E))
    W = s[:, None] * E * s[None, :]
    Winv_ref = np.linalg.inv(W)
    Winv = X / s[:, None] / s[None, :]
    kappa = np.linalg.cond(W)
    err = np.linalg.norm(Winv - Winv_ref, 2) / np.linalg.norm(Winv_ref, 2)
    assert err <= 10 * n * 2.0 ** -24 * kappa, (err, kappa)
    assert np.linalg.eigvalsh(Winv).min() > 0


def test_coarse_inverse_rejects_a_non_positive_pivot(mor):
    import torch
    E = _spd(70, 3)
    E[5, 5] = -1.0
    with pytest.raises(mor.MorError):
        mor.coarse_inverse(torch.as_tensor(E, device="cuda"))


def test_finer_aggregates_cut_iterations_not_results(mor):
    mesh, kappa, owner, p = synth.workload("cube64_p4")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    out = {}
    for rows in (100, 35):
        b = mor.Bases(sd, mor.basis_opts(rank=p["rank"], oversample=p["oversample"],
                                         seed=p["seed"], precision="mixed", cg_rtol=1e-9,
                                         coarse_rows=rows))
        assert b.converged
        x, info = mor.Reduced(sd, b).solve(rtol=1e-12)
        out[rows] = (b.stats(), b.sigma(), info["energy"])
    it100, it35 = out[100][0][:4], out[35][0][:4]
    assert it35.sum() <= 0.9 * it100.sum(), (it100, it35)
    s100, s35 = out[100][1], out[35][1]
    assert np.max(np.abs(s35 - s100)) <= 1e-7 * s100.max()
    assert abs(out[35][2] - out[100][2]) <= 1e-8 * out[100][2]


def test_tensor_core_coarse_product_matches_simt(mor):
    # tc_gram 1 forms y_c = E^{-1} r_c on the tensor cores (bf16 high and low parts,
    # three products), tc_gram 0 in binary32 SIMT: the preconditioners differ at the
    # 1e-5 level, which may move an iteration count by one check interval (8) but not
    # the bases beyond the CG tolerance
    mesh, kappa, owner, p = synth.workload("cube64_p4")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    out = {}
    for tc in (0, 1):
        b = mor.Bases(sd, mor.basis_opts(rank=p["rank"], oversample=p["oversample"],
                                         seed=p["seed"], precision="mixed", cg_rtol=1e-9,
                                         tc_gram=tc))
        assert b.converged
        x, info = mor.Reduced(sd, b).solve(rtol=1e-12)
        out[tc] = (b.stats(), b.sigma(), info["energy"])
    it0, it1 = out[0][0][:4], out[1][0][:4]
    assert np.all(np.abs(it1 - it0) <= 8), (it0, it1)
    assert np.max(np.abs(out[1][1] - out[0][1])) <= 1e-7 * out[0][1].max()
    assert abs(out[1][2] - out[0][2]) <= 1e-8 * out[0][2]


def test_binary64_coarse_levels_agree(mor):
    # the binary64 path's SIMT coarse product with one row per thread (300-row
    # aggregates, at most 256 per subdomain) and two rows per thread (35-row aggregates,
    # about 1,000): different preconditioners, the same solutions to the CG tolerance
    mesh, kappa, owner, p = synth.workload("cube64_p4")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    out = {}
    for rows in (300, 35):
        b = mor.Bases(sd, mor.basis_opts(rank=p["rank"], oversample=p["oversample"],
                                         seed=p["seed"], precision="fp64", cg_rtol=1e-11,
                                         coarse_rows=rows))
        assert b.converged
        x, info = mor.Reduced(sd, b).solve(rtol=1e-12)
        out[rows] = (b.stats(), b.sigma(), info["energy"])
    assert out[35][0][:4].sum() < out[300][0][:4].sum()
    assert np.max(np.abs(out[35][1] - out[300][1])) <= 1e-9 * out[300][1].max()
    assert abs(out[35][2] - out[300][2]) <= 1e-9 * out[300][2]
