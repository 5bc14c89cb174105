"""Paper-literal weights on the GPU against the oracle on the 16^3 cube (8 subdomains,
|I| + |B| = 1,728..2,197, |B| = 397..469).

- R_BB (Lemma 4.1): the trailing block of the Cholesky factor of H^+ in [I; B] order,
  B in ascending node order, from the GPU's batched dense Cholesky, against the oracle's
  dense LAPACK factor (rbb_cholesky).  Both are the unique Cholesky factor of the same
  Schur complement, so they agree to rounding: 1e-10 of the largest entry.
- The paper's sketch W = R_BB^{-1} S (Sec. 6, S Gaussian on B with the oracle's Philox
  counters): singular values within 1e-10 sigma_1, subspaces within 1e-10 / gap, and the
  reduced energy within 1e-10, as for the field sketch.
- The explicit weighted SVD of Eq. (14), R_i Z_i R_BB^{-1} with dense factors of A_II,
  H_i and H^+: the GPU takes the singular values from eig(X^T X), so sigma_j carries an
  absolute error of about u sigma_1^2 / sigma_j (u = 2^-53); the leading 3 m singular
  values are compared within 1e-10 sigma_1, the basis within 1e-10 / gap, and the
  reduced energy and solution within 1e-10 of the oracle's.
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


def _sin_max(Qg, Qo, A):
    R = Qg - Qo @ (Qo.T @ (A @ Qg))
    return np.sqrt(max(0.0, np.linalg.eigvalsh(R.T @ (A @ R)).max()))


def _check(mor, cube16, b, ref, nsig):
    mesh, kappa, owner, p, sd = cube16
    m = p["rank"]
    sig = b.sigma()
    for i, ob in enumerate(ref["bases"]):
        s = ob["sigma"]
        n = min(nsig, len(s))
        assert np.max(np.abs(sig[i, :n] - s[:n])) <= 1e-10 * s[0], i
        Qg = b.Q(i)[:, :b.kept[i]]
        assert Qg.shape[1] == ob["Q"].shape[1], i
        gap = (s[m - 1] - s[m]) / s[0]
        assert _sin_max(Qg, ob["Q"], ob["A_PP"]) <= 1e-10 / min(1.0, gap), i
    r = mor.Reduced(sd, b)
    x, info = r.solve(rtol=1e-14)
    assert info["converged"]
    assert abs(info["energy"] - ref["E"]) <= 1e-10 * ref["E"]
    u = mor.lift(sd, b, x).cpu().numpy()
    assert reduced.energy_norm(mesh, kappa, u - ref["u_red"]) <= \
        1e-10 * reduced.energy_norm(mesh, kappa, ref["u_red"])


def test_rbb_from_batched_dense_cholesky(mor, cube16):
    mesh, kappa, owner, p, sd = cube16
    b = mor.Bases(sd, mor.basis_opts(rank=p["rank"], oversample=p["oversample"], seed=p["seed"],
                                     precision="fp64", cg_rtol=1e-13, sketch="paper"))
    assert b.converged
    for i in range(sd.n_sub):
        s = osub.subdomain_sets(mesh, owner, i, p["r_hops"])
        loc = obasis.local_system(mesh, kappa, s)
        ref = obasis.rbb_cholesky(loc["H_plus"], loc["nI"])
        got = b.rbb(i)
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref)), i
        assert np.all(np.tril(got, -1) == 0.0)


def test_paper_sketch_matches_oracle(mor, cube16):
    mesh, kappa, owner, p, sd = cube16
    ref = pipeline.run(mesh, kappa, owner, p["rank"], p["oversample"], p["r_hops"], p["seed"],
                       sketch="paper", fe_solution=False)
    b = mor.Bases(sd, mor.basis_opts(rank=p["rank"], oversample=p["oversample"], seed=p["seed"],
                                     precision="fp64", cg_rtol=1e-13, sketch="paper"))
    assert b.converged
    _check(mor, cube16, b, ref, p["rank"] + p["oversample"])


def test_explicit_weighted_svd_matches_oracle(mor, cube16):
    mesh, kappa, owner, p, sd = cube16
    ref = pipeline.run(mesh, kappa, owner, p["rank"], 0, p["r_hops"], p["seed"], explicit=True,
                       fe_solution=False)
    b = mor.Bases(sd, mor.basis_opts(rank=p["rank"], oversample=0, seed=p["seed"],
                                     precision="fp64", explicit_svd=1))
    assert b.k == sd.counts[:, 1].max()
    _check(mor, cube16, b, ref, 3 * p["rank"])
    # the randomized bases approximate the explicit (optimal) ones: their singular values
    # never exceed the explicit ones (projection, interlacing)
    br = mor.Bases(sd, mor.basis_opts(rank=p["rank"], oversample=p["oversample"],
                                      seed=p["seed"], precision="fp64", cg_rtol=1e-13))
    sr, se = br.sigma(), b.sigma()
    k = sr.shape[1]
    assert np.all(sr <= se[:, :k] * (1 + 1e-10))


def test_explicit_svd_in_tolerance_mode(mor, cube16):
    # Eq. (15) with the explicit SVD: keep sigma_j > eps; eps in a clear gap of the
    # oracle's spectrum, so the kept counts must agree
    mesh, kappa, owner, p, sd = cube16
    pre = pipeline.run(mesh, kappa, owner, 1, 0, p["r_hops"], p["seed"], explicit=True,
                       fe_solution=False)
    s = np.sort(np.concatenate([b["sigma"][:60] for b in pre["bases"]]))[::-1]
    gaps = [j for j in range(len(s) - 1) if s[j] > 1.05 * s[j + 1]]
    j = min(gaps, key=lambda g: abs(np.log(np.sqrt(s[g] * s[g + 1]) / 1e-2)))
    eps = float(np.sqrt(s[j] * s[j + 1]))
    ref = pipeline.run(mesh, kappa, owner, 1, 0, p["r_hops"], p["seed"], explicit=True,
                       eps=eps, fe_solution=False)
    b = mor.Bases(sd, mor.basis_opts(rank=1, oversample=0, seed=p["seed"], precision="fp64",
                                     explicit_svd=1, eps=eps))
    assert np.array_equal(b.kept, [ob["n_kept"] for ob in ref["bases"]])
    r = mor.Reduced(sd, b)
    x, info = r.solve(rtol=1e-14)
    assert abs(info["energy"] - ref["E"]) <= 1e-10 * ref["E"]
