"""Tensor-core Grams (tcgen05, mor_tc.cu) against binary64.

The mixed path forms its dense contractions (X^T H_i X, G_B of Eq. (24), V^T A V, and the
interface blocks of Eq. (23)) on the tensor cores from exact 7-bit integer slices of the
binary64 operands, scaled per column.  The only error is the slicing: each operand entry
is kept to 2^-29 of its column's largest entry (four slices of 7 bits below a leading
bit), so entry (i, j) of X^T Y is off by at most about 2^-28 rows max|X_i| max|Y_j| and,
for random data, by about sqrt(rows) times that.  The checks use the worst-case bound
2^-26 rows max|X_i| max|Y_j|, on graded columns (norms spread over twelve orders of
magnitude, as the sketch columns of G_B are), row counts that are not multiples of the
32-row MMA block and that cross the 256-row accumulator flush, one column, 128 columns
and zero columns.  The mixed path with tensor-core Grams (tc_gram 1: the H_i-Grams and
G_B; tc_gram 2: the interface blocks of Eq. (23) too) stays within 1e-6 relative energy
of the binary64 path and within 1e-7 of the mixed path with binary64 Grams (the mixed
local solves stop at 1e-9, so both mixed bases are perturbed at about that level).  With
tc_gram 2 the Galerkin identity x^T K~ x = ||Q x||_A^2 holds only to the slicing error of
the interface blocks; on this unit-coefficient mesh that is below 1e-7 relative.
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


@pytest.mark.parametrize("rows,nx,ny", [(1000, 44, 44), (31, 7, 13), (257, 1, 128),
                                        (5000, 128, 36), (0, 4, 4)])
def test_tc_gram_error_bound(mor, rows, nx, ny):
    import torch
    rng = np.random.default_rng(rows + nx + ny)
    X = rng.standard_normal((rows, nx)) * np.logspace(0, -12, nx)[None, :]
    Y = rng.standard_normal((rows, ny)) * np.logspace(-3, 3, ny)[None, :]
    if nx > 2:
        X[:, 2] = 0.0                        # a zero column
    G = mor.tc_gram(torch.as_tensor(X, device="cuda"), torch.as_tensor(Y, device="cuda"))
    G = G.cpu().numpy()
    ref = X.T @ Y
    bound = 2.0 ** -26 * max(rows, 1) * np.outer(np.abs(X).max(axis=0, initial=0.0),
                                                np.abs(Y).max(axis=0, initial=0.0))
    assert np.all(np.abs(G - ref) <= bound)
    if rows >= 1000:
        # graded accuracy: every entry relative to its own column norms, not the largest
        nrm = np.outer(np.linalg.norm(X, axis=0), np.linalg.norm(Y, axis=0))
        ok = nrm > 0
        assert np.max(np.abs(G - ref)[ok] / nrm[ok]) < 1e-7


def test_tc_gram_level_out_of_range(mor):
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    with pytest.raises(mor.MorError):
        mor.Bases(sd, mor.basis_opts(rank=4, precision="mixed", tc_gram=3))


def test_mixed_path_with_tensor_core_grams(mor):
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, p["r_hops"])
    out = {}
    for name, kw in (("fp64", dict(precision="fp64", cg_rtol=1e-13)),
                     ("mixed_tc", dict(precision="mixed", cg_rtol=1e-9, tc_gram=1)),
                     ("mixed_tc2", dict(precision="mixed", cg_rtol=1e-9, tc_gram=2)),
                     ("mixed_fp64", dict(precision="mixed", cg_rtol=1e-9, tc_gram=0))):
        b = mor.Bases(sd, mor.basis_opts(rank=p["rank"], oversample=p["oversample"],
                                         seed=p["seed"], **kw))
        r = mor.Reduced(sd, b)
        x, info = r.solve(rtol=1e-13)
        assert info["converged"], name
        out[name] = (b, mor.lift(sd, b, x), info)
    u64 = out["fp64"][1]
    n64 = mor.energy_norm(sd, u64)
    assert mor.energy_norm(sd, out["mixed_tc"][1], u64) / n64 <= 1e-6
    assert mor.energy_norm(sd, out["mixed_tc"][1], out["mixed_fp64"][1]) / n64 <= 1e-7
    assert mor.energy_norm(sd, out["mixed_tc2"][1], u64) / n64 <= 1e-6
    # tc_gram 1 and 2 build their bases alike; only K~ differs
    s_tc2 = out["mixed_tc2"][0].sigma()
    assert np.max(np.abs(s_tc2 - out["mixed_tc"][0].sigma())) <= 1e-8 * s_tc2.max()
    b2, u2, info2 = out["mixed_tc2"]
    e2 = mor.energy_norm(sd, u2) ** 2
    assert abs(e2 - info2["energy"]) <= 1e-7 * info2["energy"]
    s_tc, s_64 = out["mixed_tc"][0].sigma(), out["mixed_fp64"][0].sigma()
    assert np.max(np.abs(s_tc - s_64)) <= 1e-8 * s_64.max()
