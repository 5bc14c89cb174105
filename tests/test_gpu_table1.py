"""The behaviour of the paper's scaling tests (Sec. 7.1, Table 1 and Table 2) on the GPU:
sketch size k_i = floor(M_i / 8), tolerance eps = 1e-2, unit coefficient, r-hop
extensions, on Kuhn cubes with seeded k-means partitions standing in for the paper's
METIS partitions of its cases 4-6:

  case  paper dim V / subdomains / hops      here (n^3 cells, interior nodes)
  4     4,233 / 6 / 4                         17^3: 4,096 / 6 / 4
  5     30,481 / 30 / 5                       32^3: 29,791 / 30 / 5
  6     230,945 / 100 / 6                     62^3: 226,981 / 100 / 6

The library's load is f = 1; the paper's polynomial load gives the same reduction
error within 4% at case 4 (oracle: 1.24e-4 against 1.20e-4).  The paper reports
reduction errors ||grad(u - u~)|| of 9.0e-5, 2.1e-4, 2.6e-4 (Table 1) and
dim V~ / dim V of 4.2%, 4.7%, 3.0% (Table 2) for cases 4-6.  The checks: dim V~ / dim V lies
within a factor 2 of the paper's, the relative reduction error against the unreduced FE
solution (the oracle's global system) stays below 5e-3, and the mixed path reaches the
binary64 path's reduced solution (within 1e-6 relative energy).  The randomized bases
are less accurate than the paper's at the smallest sketches: at case 4 (k_i = 42..66)
the error is about 3e-3 against the explicit SVD's 1.2e-4 for the same partition, and
it falls towards the paper's values as the sketches widen (cases 5-6).  Case 4 also
runs the explicit SVD (Eq. (14)) on the GPU.  Run with -s to print the measured rows.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.linalg import cg

import synth
from oracle import fem

pytestmark = pytest.mark.gpu

CASES = [  # case, cells per side, subdomains, hops, paper dim V~ / dim V, paper red. error
    (4, 17, 6, 4, 178 / 4233, 9.0e-5),
    (5, 32, 30, 5, 1436 / 30481, 2.1e-4),
    (6, 62, 100, 6, 6880 / 230945, 2.6e-4),
]


@pytest.fixture(scope="module")
def mor():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2404_06260_gb300 import _build
    _build.build()
    from paper_2404_06260_gb300 import mor as m
    return m


@pytest.mark.parametrize("case,n,parts,hops,ratio_paper,err_paper", CASES)
def test_scaling_case(mor, case, n, parts, hops, ratio_paper, err_paper):
    import torch
    mesh = synth.kuhn_cube(n)
    owner = synth.kmeans_owner(mesh, parts, 1000 + n)
    kappa = np.ones(mesh.n_tets)
    gm = mor.Mesh(mesh.xyz, mesh.tets, kappa, mesh.dirichlet)
    sd = mor.Subdomains(gm, owner, hops)
    assert sd.n_sub == parts
    # the unreduced FE solution: the oracle's global system, solved by Jacobi-
    # preconditioned CG to a relative residual of 1e-13 (a sparse direct solve of the
    # 227k-unknown case takes minutes on the host); the energy error of that solve is
    # far below the 1e-4 reduction errors measured
    A, b, fmap, free = fem.global_system(mesh, kappa)
    A = A.tocsr()
    M = sp.diags(1.0 / A.diagonal())
    try:
        uf, info = cg(A, b, rtol=1e-13, atol=0.0, maxiter=20000, M=M)
    except TypeError:
        uf, info = cg(A, b, tol=1e-13, atol=0.0, maxiter=20000, M=M)
    assert info == 0
    assert np.linalg.norm(b - A @ uf) <= 1e-12 * np.linalg.norm(b)
    u = np.zeros(mesh.n_nodes)
    u[free] = uf
    u_d = torch.as_tensor(u, device="cuda")
    dim_v = int(free.size)
    rows = {}
    for prec, rt in (("fp64", 1e-11), ("mixed", 1e-9)):
        bases = mor.Bases(sd, mor.basis_opts(rank=1, oversample=0, seed=7, precision=prec,
                                             cg_rtol=rt, eps=1e-2, sketch_div=8))
        assert bases.converged, prec
        red = mor.Reduced(sd, bases)
        x, info = red.solve(rtol=1e-12)
        assert info["converged"], prec
        ut = mor.lift(sd, bases, x)
        err = mor.energy_norm(sd, ut, u_d) / mor.energy_norm(sd, u_d)
        rows[prec] = (bases.total_kept, err, ut, bases.k)
    kept, err, ut, k = rows["mixed"]
    ratio = kept / dim_v
    print("\ncase %d: dim V %d, dim V~ %d (%.2f%%; paper %.2f%%), widest sketch %d, "
          "reduction error %.2e (binary64 %.2e; paper %.1e)"
          % (case, dim_v, kept, 100 * ratio, 100 * ratio_paper, k, err, rows["fp64"][1],
             err_paper))
    assert err < 5e-3 and rows["fp64"][1] < 5e-3
    assert 0.5 * ratio_paper < ratio < 2.0 * ratio_paper
    e = mor.energy_norm(sd, ut, rows["fp64"][2]) / mor.energy_norm(sd, rows["fp64"][2])
    assert e <= 1e-6, e
    if case == 4:
        # the explicit weighted SVD (Eq. (14)) with the same eps
        bx = mor.Bases(sd, mor.basis_opts(rank=1, oversample=0, seed=7, precision="fp64",
                                          eps=1e-2, explicit_svd=1))
        rx = mor.Reduced(sd, bx)
        xx, infox = rx.solve(rtol=1e-12)
        ux = mor.lift(sd, bx, xx)
        errx = mor.energy_norm(sd, ux, u_d) / mor.energy_norm(sd, u_d)
        print("case 4, explicit SVD: dim V~ %d (%.2f%%), reduction error %.2e"
              % (bx.total_kept, 100 * bx.total_kept / dim_v, errx))
        assert errx < 1e-3
