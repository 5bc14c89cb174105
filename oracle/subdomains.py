"""Overlapping subdomains and their extensions (Sec. 3; Sec. 6 step 1; Sec. 7.1).

Given node owner labels (the graph partition of Sec. 6 step 1):
  P_i        nodes owned by subdomain i;
  omega_i    elements with at least one node in P_i (Fig. 1 caption: "elements that
             have at least one node belonging to a specific subgraph"); two subdomains
             then overlap in one layer of elements;
  ball       nodes within r mesh-edge hops of P_i (the r-hops of Sec. 7.1);
  T_i^+      elements touching the ball (so every ball node is interior to omega_i^+);
  I          free nodes of T_i^+ whose incident elements all lie in T_i^+ (interior
             of omega_i^+, Sec. 4), B = the other free nodes of T_i^+ (on
             d omega_i^+ minus d Omega);
  omega DOFs free nodes of omega_i (the space V_i);
  owned      free nodes of P_i: the nodes kept by the stitching restriction D_i.
Hops run over the edges of the tetrahedra (every pair of vertices of an element).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def node_adjacency(tets, n_nodes):
    r = np.repeat(tets, 4, axis=1).ravel()
    c = np.tile(tets, (1, 4)).ravel()
    A = sp.coo_matrix((np.ones(len(r), dtype=np.int8), (r, c)), shape=(n_nodes, n_nodes))
    return A.tocsr()


def hops_for(n_owned, r_hops):
    """r_hops, or for r_hops = -1 about half the subdomain width:
    max(1, round(n_owned^(1/3) / 2)) (halves round up), so the extension roughly
    doubles the diameter (Sec. 7.1)."""
    if r_hops > 0:
        return r_hops
    return max(1, int(np.floor(np.cbrt(float(n_owned)) / 2.0 + 0.5)))


def subdomain_sets(mesh, owner, i, r_hops, adj=None):
    n = mesh.n_nodes
    tets = mesh.tets
    if adj is None:
        adj = node_adjacency(tets, n)
    P = owner == i
    ball = P.copy()
    for _ in range(hops_for(int(P.sum()), r_hops)):
        ball = ball | ((adj @ ball.astype(np.int8)) > 0)
    plus_t = np.flatnonzero(ball[tets].any(axis=1))
    omega_t = np.flatnonzero(P[tets].any(axis=1))
    cnt_all = np.bincount(tets.ravel(), minlength=n)
    cnt_plus = np.bincount(tets[plus_t].ravel(), minlength=n)
    in_plus = cnt_plus > 0
    interior = in_plus & (cnt_plus == cnt_all)
    free = mesh.dirichlet == 0
    I = np.flatnonzero(interior & free)
    B = np.flatnonzero(in_plus & ~interior & free)
    in_omega = np.bincount(tets[omega_t].ravel(), minlength=n) > 0
    omega = np.flatnonzero(in_omega & free)
    owned = np.flatnonzero(P & free)
    if not np.all(interior[omega]):
        raise ValueError("omega_i is not interior to omega_i^+ (need r_hops >= 1)")
    return dict(i=i, I=I, B=B, omega=omega, owned=owned, plus_tets=plus_t,
                omega_tets=omega_t)


def subdomain_sets_region(mesh, owner, i, r_hops, region_tets):
    """subdomain_sets computed from a candidate subset of the elements (global ids),
    for meshes too large for a global adjacency.  The candidates must include every
    element with a vertex within r + 1 edge hops of P_i: then the hop ball, T_i^+, the
    element counts that split I from B, omega_i and the owned nodes are those of the
    whole mesh, and the result equals subdomain_sets (global node and element ids)."""
    region_tets = np.asarray(region_tets, dtype=np.int64)
    T = mesh.tets[region_tets]
    nodes, loc = np.unique(T, return_inverse=True)
    loc = loc.reshape(T.shape)
    nl = len(nodes)
    P = owner[nodes] == i
    if int(P.sum()) != int(np.count_nonzero(owner == i)):
        raise ValueError("region does not contain every owned node")
    r = np.repeat(loc, 4, axis=1).ravel()
    c = np.tile(loc, (1, 4)).ravel()
    adj = sp.coo_matrix((np.ones(len(r), dtype=np.int8), (r, c)), shape=(nl, nl)).tocsr()
    ball = P.copy()
    for _ in range(hops_for(int(P.sum()), r_hops)):
        ball = ball | ((adj @ ball.astype(np.int8)) > 0)
    plus_l = np.flatnonzero(ball[loc].any(axis=1))
    omega_l = np.flatnonzero(P[loc].any(axis=1))
    cnt_all = np.bincount(loc.ravel(), minlength=nl)
    cnt_plus = np.bincount(loc[plus_l].ravel(), minlength=nl)
    in_plus = cnt_plus > 0
    interior = in_plus & (cnt_plus == cnt_all)
    free = mesh.dirichlet[nodes] == 0
    in_omega = np.bincount(loc[omega_l].ravel(), minlength=nl) > 0
    if not np.all(interior[in_omega & free]):
        raise ValueError("omega_i is not interior to omega_i^+ (need r_hops >= 1)")
    # global ids ascending: nodes are sorted, and so are the candidate element ids
    pl = np.sort(region_tets[plus_l])
    ol = np.sort(region_tets[omega_l])
    return dict(i=i, I=nodes[interior & free], B=nodes[in_plus & ~interior & free],
                omega=nodes[in_omega & free], owned=nodes[P & free], plus_tets=pl,
                omega_tets=ol)


def all_subdomains(mesh, owner, r_hops):
    adj = node_adjacency(mesh.tets, mesh.n_nodes)
    n_sub = int(owner.max()) + 1
    return [subdomain_sets(mesh, owner, i, r_hops, adj) for i in range(n_sub)]


def interface_tets(mesh, owner):
    """omega_0: elements shared by at least two subdomains omega_i, i.e. elements whose
    vertices have at least two different owners (Sec. 6 step 3)."""
    o = owner[mesh.tets]
    return np.flatnonzero(np.any(o != o[:, :1], axis=1))
