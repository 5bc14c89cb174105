"""P1 tetrahedral finite elements (Sec. 2, Prob. "dweak"; Sec. 4 inner products).

Element quantities for a tetrahedron T with vertices x_0..x_3:
  barycentric gradients  G = [grad lambda_a]: with J = [x_1-x_0, x_2-x_0, x_3-x_0],
                         grad lambda_a = row (a-1) of J^{-1} (a = 1..3),
                         grad lambda_0 = -(sum of the other three);
  volume                 |T| = det(J) / 6;
  stiffness              K_T[a,b] = k_T |T| grad lambda_a . grad lambda_b
                         (bilinear form of -div(k grad u); k = 1 is the paper's model problem, Eq. (1));
  mass                   M_T[a,b] = |T| (1 + delta_ab) / 20;
  H1 inner product       K_T(k = 1) + M_T  (the forms of Sec. 4 defining R_i and R_BB);
  load                   int_T f lambda_a; for f = 1 this is |T| / 4.
Assembly sums element matrices into sparse matrices with SciPy (duplicate COO entries
are summed).  Node maps send global node ids to local indices, -1 = not a DOF.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.special import roots_jacobi


def tet_geometry(xyz, tets):
    """Barycentric gradients (n_t, 4, 3) and volumes (n_t,).  Raises on det <= 0."""
    X = xyz[tets]                                   # (t, 4, 3)
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))  # columns = edges
    det = np.linalg.det(J)
    if np.any(det <= 0):
        raise ValueError("non-positive tetrahedron volume")
    Jinv = np.linalg.inv(J)
    G = np.empty((len(tets), 4, 3))
    G[:, 1:, :] = Jinv
    G[:, 0, :] = -Jinv.sum(axis=1)
    return G, det / 6.0


def stiffness_elements(G, vol, kappa=None):
    K = np.einsum("tai,tbi->tab", G, G) * vol[:, None, None]
    if kappa is not None:
        K = K * kappa[:, None, None]
    return K


def mass_elements(vol):
    M = np.full((len(vol), 4, 4), 1.0) + np.eye(4)[None]
    return M * (vol / 20.0)[:, None, None]


def assemble_matrix(tets, Ke, row_map, n_rows, col_map=None, n_cols=None):
    """Sum element matrices Ke (n_t, 4, 4) over tets into an n_rows x n_cols CSR matrix,
    keeping entries whose row and column both map to a DOF."""
    if col_map is None:
        col_map, n_cols = row_map, n_rows
    R = row_map[tets]                      # (t, 4)
    C = col_map[tets]
    rows = np.broadcast_to(R[:, :, None], Ke.shape).ravel()
    cols = np.broadcast_to(C[:, None, :], Ke.shape).ravel()
    vals = Ke.ravel()
    keep = (rows >= 0) & (cols >= 0)
    A = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n_rows, n_cols))
    return A.tocsr()


def assemble_vector(tets, fe, row_map, n_rows):
    """Sum element vectors fe (n_t, 4) into a length-n_rows vector."""
    R = row_map[tets].ravel()
    v = fe.ravel()
    keep = R >= 0
    return np.bincount(R[keep], weights=v[keep], minlength=n_rows)


def load_unit(vol):
    """int_T 1 * lambda_a = |T|/4."""
    return np.repeat((vol / 4.0)[:, None], 4, axis=1)


def tet_quadrature(order_pts: int = 3):
    """Conical-product Gauss-Jacobi rule on the reference tetrahedron (Stroud):
    x = u, y = v (1-u), z = w (1-u)(1-v), Jacobian (1-u)^2 (1-v), Gauss-Jacobi in u
    (weight (1-u)^2), v (weight (1-v)) and Gauss-Legendre in w, each with order_pts
    points on [0, 1].  Exact for polynomials of degree <= 2*order_pts - 1.
    Returns reference barycentric points (n_q, 4) and weights summing to 1/6."""
    def gj(n, alpha):
        x, w = roots_jacobi(n, alpha, 0.0)       # on [-1,1], weight (1-x)^alpha
        t = (x + 1.0) / 2.0
        return t, w / 2.0 ** (alpha + 1)
    u, wu = gj(order_pts, 2.0)
    v, wv = gj(order_pts, 1.0)
    w, ww = gj(order_pts, 0.0)
    U, V, W = np.meshgrid(u, v, w, indexing="ij")
    WT = wu[:, None, None] * wv[None, :, None] * ww[None, None, :]
    x = U
    y = V * (1 - U)
    z = W * (1 - U) * (1 - V)
    lam = np.stack([1 - x - y - z, x, y, z], axis=-1).reshape(-1, 4)
    return lam, WT.ravel()


def load_function(xyz, tets, vol, f, order_pts: int = 3):
    """int_T f lambda_a by the conical-product rule (exact to degree 2*order_pts-1)."""
    lam, wq = tet_quadrature(order_pts)
    X = xyz[tets]                                        # (t, 4, 3)
    pts = np.einsum("qa,tai->tqi", lam, X)              # (t, q, 3)
    fv = f(pts[..., 0], pts[..., 1], pts[..., 2])       # (t, q)
    return 6.0 * vol[:, None] * np.einsum("tq,q,qa->ta", fv, wq, lam)


def free_map(dirichlet):
    """Global node -> free-DOF index (-1 on the Dirichlet boundary)."""
    m = -np.ones(len(dirichlet), dtype=np.int64)
    free = np.flatnonzero(dirichlet == 0)
    m[free] = np.arange(len(free))
    return m, free


def global_system(mesh, kappa, f=None):
    """Global stiffness A and load b on the free DOFs (Prob. "dweak")."""
    G, vol = tet_geometry(mesh.xyz, mesh.tets)
    fmap, free = free_map(mesh.dirichlet)
    A = assemble_matrix(mesh.tets, stiffness_elements(G, vol, kappa), fmap, len(free))
    fe = load_unit(vol) if f is None else load_function(mesh.xyz, mesh.tets, vol, f)
    b = assemble_vector(mesh.tets, fe, fmap, len(free))
    return A, b, fmap, free
