"""The whole hot path on one mesh: subdomains -> local bases -> projection -> reduced
solve (Sec. 6 steps 1-3), plus the unreduced FE solution for error measurements."""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import splu

from . import fem
from .basis import local_basis
from .reduced import (energy_norm, lift, project_explicit, project_interface,
                      solve_reduced, stitched_Q)
from .subdomains import all_subdomains


def run(mesh, kappa, owner, rank, oversample, r_hops, seed, sketch="field",
        explicit=False, eps=None, tau=1e-12, f=None, keep_all=False, fe_solution=True,
        interface=True, h1_weighted=False):
    subs = all_subdomains(mesh, owner, r_hops)
    ranks = np.broadcast_to(np.asarray(rank), (len(subs),))   # per-subdomain m_i
    bases = [local_basis(mesh, kappa, s, int(ranks[j]), oversample, seed, sketch=sketch,
                         explicit=explicit, eps=eps, tau=tau, f=f, keep_all=keep_all,
                         h1_weighted=h1_weighted)
             for j, s in enumerate(subs)]
    out = dict(subs=subs, bases=bases)
    if interface:
        K, bt, pairs = project_interface(mesh, kappa, owner, bases)
        out["pairs"] = pairs
    else:
        A, b, _, _ = fem.global_system(mesh, kappa, f)
        K, bt = project_explicit(A, b, stitched_Q(mesh, bases))
    x, E = solve_reduced(K, bt)
    out.update(K=K, bt=bt, x=x, E=E, u_red=lift(mesh, bases, x))
    if fe_solution:
        A, b, fmap, free = fem.global_system(mesh, kappa, f)
        u_free = splu(A.tocsc()).solve(b)
        u = np.zeros(mesh.n_nodes)
        u[free] = u_free
        out["u"] = u
        out["E_fe"] = float(b @ u_free)
        out["red_err"] = energy_norm(mesh, kappa, u - out["u_red"]) / energy_norm(mesh, kappa, u)
    return out
