"""The paper's sketch size k_i = floor(M_i / 8) with tolerance-mode truncation (Sec. 7.1,
App. C, Eq. (15)) on the 16^3 cube, against the oracle.

mor_basis_opts.sketch_div = d sketches k_i = max(1, floor(|B_i| / d)) columns per
subdomain and keeps the sigma_j > eps among them.  With d = 8 (the paper's rule) the
16^3 subdomains sketch 38..58 columns (the small dense kernels); with d = 4 they sketch
76..117 (the widest sketch sets the column count of the batch, so the wide Gram,
Jacobi and row-product kernels run).  eps is placed in the
middle of a clear gap (ratio > 1.05) of the oracle's singular values near 1e-2, so the
binary64 path must keep the same number of directions in every subdomain.

Tolerances as for the 16^3 parity tests: singular values within 1e-10 sigma_1, kept
subspaces within 1e-8 (principal-angle sines in the A[P_i, P_i] inner product; the cut
lies in a gap of >= 5%), reduced energy and lifted solution within 1e-10; the mixed path
within 1e-6 relative energy of the binary64 path.
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
def cube16(mor):
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    return mesh, kappa, owner, p, sd


def _eps_in_gap(sigmas, target=1e-2):
    s = np.sort(np.concatenate(sigmas))[::-1]
    gaps = [j for j in range(len(s) - 1) if s[j] > 1.05 * s[j + 1] and s[j + 1] > 0]
    j = min(gaps, key=lambda g: abs(np.log(np.sqrt(s[g] * s[g + 1]) / target)))
    return float(np.sqrt(s[j] * s[j + 1]))


@pytest.mark.parametrize("div", [8, 4])
def test_paper_sketch_size_in_tolerance_mode(mor, cube16, div):
    mesh, kappa, owner, p, sd = cube16
    kk = np.maximum(1, sd.counts[:, 1] // div)
    if div == 8:
        assert kk.max() <= 79          # the small dense kernels
    else:
        assert kk.max() > 80           # the wide kernels (the widest sketch sets kp)
    # eps in a gap of the oracle's spectrum near 1e-2
    pre = pipeline.run(mesh, kappa, owner, kk, 0, p["r_hops"], p["seed"], fe_solution=False)
    eps = _eps_in_gap([b["sigma"] for b in pre["bases"]])
    ref = pipeline.run(mesh, kappa, owner, kk, 0, p["r_hops"], p["seed"], eps=eps,
                       fe_solution=False)
    out = {}
    for prec, rt in (("fp64", 1e-13), ("mixed", 1e-9)):
        b = mor.Bases(sd, mor.basis_opts(rank=1, oversample=0, seed=p["seed"], precision=prec,
                                         cg_rtol=rt, eps=eps, sketch_div=div))
        assert b.converged, prec
        assert b.k == kk.max()
        r = mor.Reduced(sd, b)
        x, info = r.solve(rtol=1e-14)
        assert info["converged"]
        out[prec] = (b, r, x, info, mor.lift(sd, b, x))
    b, r, x, info, u = out["fp64"]
    sig = b.sigma()
    assert np.array_equal(b.kept, [ob["n_kept"] for ob in ref["bases"]])
    assert b.kq == ((b.kept.max() + 3) // 4) * 4
    for i, ob in enumerate(ref["bases"]):
        n = int(kk[i])
        assert np.max(np.abs(sig[i, :n] - ob["sigma"][:n])) <= 1e-10 * ob["sigma"][0], i
        assert np.all(sig[i, n:] == 0.0)
        A = ob["A_PP"]
        Qg = b.Q(i)[:, :b.kept[i]]
        R = Qg - ob["Q"] @ (ob["Q"].T @ (A @ Qg))
        assert np.sqrt(max(0.0, np.linalg.eigvalsh(R.T @ (A @ R)).max())) < 1e-8, i
    assert abs(info["energy"] - ref["E"]) <= 1e-10 * ref["E"]
    ug = u.cpu().numpy()
    assert reduced.energy_norm(mesh, kappa, ug - ref["u_red"]) <= \
        1e-10 * reduced.energy_norm(mesh, kappa, ref["u_red"])
    um = out["mixed"][4]
    e = mor.energy_norm(sd, um, u) / mor.energy_norm(sd, u)
    assert e <= 1e-6, e


def test_sketch_div_argument_checks(mor, cube16):
    mesh, kappa, owner, p, sd = cube16
    with pytest.raises(mor.MorError):
        mor.Bases(sd, mor.basis_opts(rank=1, oversample=0, seed=1, sketch_div=8))  # no eps
    with pytest.raises(mor.MorError):
        mor.Bases(sd, mor.basis_opts(rank=1, oversample=0, seed=1, eps=1e-2, sketch_div=-1))
