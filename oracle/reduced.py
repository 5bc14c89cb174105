"""Stitching, projection and the reduced solve (Eq. (11), Def. 3.1, Eq. (23),
Sec. 6 step 3).

  stitched basis  the global matrix Q whose column block i holds Q_i on the owned
                  nodes P_i and zero elsewhere (the stitching operator S_i keeps the
                  nodal values of omega_i minus d omega_i and extends by zero; with
                  owned nodes as that interior every node is kept by exactly one i,
                  so sum_i S_i(v|omega_i) = v);
  explicit        K~ = Q^T A Q, b~ = Q^T b with the assembled global A;
  interface-only  K~_ii from step 2, K~_ij (i != j) = Q_i^T A_0[P_i, P_j] Q_j with A_0
                  assembled over omega_0 only (elements shared by >= 2 subdomains);
  reduced solve   K~ x = b~ by a dense Cholesky (the paper uses diagonally
                  preconditioned CG; the oracle solves directly);
  lift            u~ = Q x.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem
from .subdomains import interface_tets


def offsets(bases):
    n = [b["Q"].shape[1] for b in bases]
    return np.concatenate([[0], np.cumsum(n)])


def stitched_Q(mesh, bases):
    fmap, free = fem.free_map(mesh.dirichlet)
    off = offsets(bases)
    r, c, v = [], [], []
    for b, o in zip(bases, off[:-1]):
        Q = b["Q"]
        rr = np.repeat(fmap[b["owned"]], Q.shape[1])
        cc = np.tile(o + np.arange(Q.shape[1]), Q.shape[0])
        r.append(rr)
        c.append(cc)
        v.append(Q.ravel())
    return sp.csr_matrix((np.concatenate(v), (np.concatenate(r), np.concatenate(c))),
                         shape=(len(free), off[-1]))


def project_explicit(A, b, Qg):
    K = (Qg.T @ (A @ Qg)).toarray()
    return 0.5 * (K + K.T), Qg.T @ b


def project_interface(mesh, kappa, owner, bases):
    """K~ from the diagonal blocks of step 2 and A_0 on omega_0 (Sec. 6 step 3)."""
    t0 = interface_tets(mesh, owner)
    T0 = mesh.tets[t0]
    G, vol = fem.tet_geometry(mesh.xyz, T0)
    fmap, free = fem.free_map(mesh.dirichlet)
    A0 = fem.assemble_matrix(T0, fem.stiffness_elements(G, vol, kappa[t0]), fmap,
                             len(free)).tocsr()
    off = offsets(bases)
    K = np.zeros((off[-1], off[-1]))
    bt = np.zeros(off[-1])
    rows_of = [fmap[b["owned"]] for b in bases]
    for i, bi in enumerate(bases):
        K[off[i]:off[i + 1], off[i]:off[i + 1]] = bi["Kii"]
        bt[off[i]:off[i + 1]] = bi["bt"]
    own_free = owner[free]
    Ac = A0.tocoo()
    oi, oj = own_free[Ac.row], own_free[Ac.col]
    pairs = set(zip(oi[oi != oj].tolist(), oj[oi != oj].tolist()))
    for i, j in sorted(pairs):
        Aij = A0[rows_of[i]][:, rows_of[j]]
        K[off[i]:off[i + 1], off[j]:off[j + 1]] = bases[i]["Q"].T @ (Aij @ bases[j]["Q"])
    return 0.5 * (K + K.T), bt, sorted(pairs)


def solve_reduced(K, bt):
    c = sla.cho_factor(K)
    x = sla.cho_solve(c, bt)
    return x, float(bt @ x)


def lift(mesh, bases, x):
    """u~ on all nodes (zero on the Dirichlet boundary)."""
    u = np.zeros(mesh.n_nodes)
    off = offsets(bases)
    for b, o0, o1 in zip(bases, off[:-1], off[1:]):
        u[b["owned"]] = b["Q"] @ x[o0:o1]
    return u


def energy_norm(mesh, kappa, v):
    """||v||_A = sqrt(sum_T v_T^T K_T v_T) over all elements, v on all nodes."""
    G, vol = fem.tet_geometry(mesh.xyz, mesh.tets)
    K = fem.stiffness_elements(G, vol, kappa)
    vt = v[mesh.tets]
    return float(np.sqrt(np.einsum("ta,tab,tb->", vt, K, vt)))
