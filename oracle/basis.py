"""Optimal local basis of one subdomain (Sec. 4 and Sec. 6 step 2), plain FP64.

Steps, in the paper's order and notation:
  1. assemble on T_i^+ the stiffness A^+ with blocks A_II, A_IB (interior I, boundary
     B), the H1 inner-product matrix H^+ (Lemma 4.2), on omega_i the H1 matrix H_i, the
     load b_I, and on the owned nodes A[P_i, P_i] and b[P_i];
  2. solve Prob. "aux1" (zero boundary, Eq. (7)): u_0 = A_II^{-1} b_I, q_0 = C_i u_0;
  3. weights: R_i = chol(H_i) (upper), R_BB = bottom-right block of chol(H^+) in [I; B]
     order (Lemma 4.1);
  4a. explicit (Eq. (14)): SVD of R_i Z_i R_BB^{-1}, Z_i = C_i A_II^{-1} A_IB;
  4b. randomized (Sec. 6, "Randomized numerical linear algebra"): sketch
      Qh Rh = R_i C_i A_II^{-1} A_IB W with W = R_BB^{-1} S_i, then the SVD of
      Qh^T R_i C_i A_II^{-1} A_IB R_BB^{-1} evaluated with two left solves (the
      transposed form of Eq. (24)); basis R_i^{-1} Qh U_m;
  5. basis V = D_i [q_0, R_i^{-1} U_m] (stitching restriction to the owned nodes,
     Def. 3.1), then the diagonal-block update: eig of K_i = V^T A[P_i,P_i] V,
     Q_i = V W Lambda^{-1/2} over eigenvalues > tau * max, so Q_i^T A_ii Q_i = I;
     projected load b~_i = Q_i^T b[P_i].

Sketch sources for W (both have columns ~ N(0, S_B^{-1}), S_B = R_BB^T R_BB):
  "paper": W = R_BB^{-1} S, S standard Gaussian on B (Philox counter (b, j, i, 1));
  "field": W = ((H^+)^{-1} L xi)_B with L = [P_T^T chol(H_T)]_T, so L L^T = H^+, and
           xi standard Gaussian per element vertex (Philox counter (T, j, i, 0)).
           Cov((H^+)^{-1} L xi) = (H^+)^{-1} and its B block is S_B^{-1} (block
           inverse of H^+), the law of R_BB^{-1} S.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
from scipy.sparse.linalg import splu

from . import fem
from .rng import field_normals, node_normals


def local_system(mesh, kappa, s, f=None, h1_weighted=False):
    """h1_weighted: the H1 forms H^+ and H_i weight their gradient part by the
    coefficient, int k grad w . grad v + w v, instead of the unweighted form of Sec. 4
    (a variant for high-contrast k; the paper analyses k = 1 only, Sec. 7.3)."""
    n = mesh.n_nodes
    I, B, omega, owned = s["I"], s["B"], s["omega"], s["owned"]
    nI, nB = len(I), len(B)
    pmap = -np.ones(n, dtype=np.int64)
    pmap[I] = np.arange(nI)
    pmap[B] = nI + np.arange(nB)
    Tp = mesh.tets[s["plus_tets"]]
    G, vol = fem.tet_geometry(mesh.xyz, Tp)
    Kp = fem.stiffness_elements(G, vol, kappa[s["plus_tets"]])
    wp = kappa[s["plus_tets"]] if h1_weighted else None
    Hp = fem.stiffness_elements(G, vol, wp) + fem.mass_elements(vol)
    A_plus = fem.assemble_matrix(Tp, Kp, pmap, nI + nB)
    H_plus = fem.assemble_matrix(Tp, Hp, pmap, nI + nB)
    fe = fem.load_unit(vol) if f is None else fem.load_function(mesh.xyz, Tp, vol, f)
    b_plus = fem.assemble_vector(Tp, fe, pmap, nI + nB)

    To = mesh.tets[s["omega_tets"]]
    Go, volo = fem.tet_geometry(mesh.xyz, To)
    wmap = -np.ones(n, dtype=np.int64)
    wmap[omega] = np.arange(len(omega))
    wo = kappa[s["omega_tets"]] if h1_weighted else None
    H_i = fem.assemble_matrix(To, fem.stiffness_elements(Go, volo, wo) + fem.mass_elements(volo),
                              wmap, len(omega))
    omap = -np.ones(n, dtype=np.int64)
    omap[owned] = np.arange(len(owned))
    A_PP = fem.assemble_matrix(To, fem.stiffness_elements(Go, volo, kappa[s["omega_tets"]]),
                               omap, len(owned))
    feo = fem.load_unit(volo) if f is None else fem.load_function(mesh.xyz, To, volo, f)
    b_P = fem.assemble_vector(To, feo, omap, len(owned))

    C = sp.csr_matrix((np.ones(len(omega)), (np.arange(len(omega)), pmap[omega])),
                      shape=(len(omega), nI))
    D = sp.csr_matrix((np.ones(len(owned)), (np.arange(len(owned)), wmap[owned])),
                      shape=(len(owned), len(omega)))
    A_plus = A_plus.tocsr()
    return dict(nI=nI, nB=nB, pmap=pmap, A_plus=A_plus, H_plus=H_plus.tocsr(), h1_w=wp,
                A_II=A_plus[:nI, :nI].tocsc(), A_IB=A_plus[:nI, nI:].tocsr(),
                b_I=b_plus[:nI], H_i=H_i, A_PP=A_PP, b_P=b_P, C=C, D=D)


def rbb_cholesky(H_plus, nI):
    """Lemma 4.1: R_BB read from the Cholesky factor of H^+ in [I; B] order."""
    Lc = np.linalg.cholesky(H_plus.toarray())
    return np.ascontiguousarray(Lc.T[nI:, nI:])


def rbb_schur(H_plus, nI):
    """Lemma 4.1 the other way: R_BB = chol(H_BB - H_BI H_II^{-1} H_IB) (upper)."""
    H = H_plus.tocsr()
    H_II = H[:nI, :nI].tocsc()
    H_IB = H[:nI, nI:]
    S = H[nI:, nI:].toarray() - H[nI:, :nI] @ splu(H_II).solve(H_IB.toarray())
    return np.linalg.cholesky(0.5 * (S + S.T)).T


def weight_rbb(H_plus, nI, dense_limit=6000):
    if H_plus.shape[0] <= dense_limit:
        return rbb_cholesky(H_plus, nI)
    return rbb_schur(H_plus, nI)


def field_sketch_rhs(mesh, s, loc, k, seed):
    """L xi on the DOFs of omega_i^+ (I then B): (nI+nB, k)."""
    T_ids = s["plus_tets"]
    Tp = mesh.tets[T_ids]
    G, vol = fem.tet_geometry(mesh.xyz, Tp)
    He = fem.stiffness_elements(G, vol, loc.get("h1_w")) + fem.mass_elements(vol)
    Le = np.linalg.cholesky(He)                          # (t, 4, 4) lower
    xi = field_normals(seed, s["i"], T_ids, k).astype(np.float64)   # (t, 4, k)
    nt = len(T_ids)
    rows = np.broadcast_to(loc["pmap"][Tp][:, :, None], (nt, 4, 4)).ravel()
    cols = (4 * np.arange(nt)[:, None, None] + np.arange(4)[None, None, :])
    cols = np.broadcast_to(cols, (nt, 4, 4)).ravel()
    vals = Le.ravel()
    keep = (rows >= 0) & (vals != 0.0)
    n_plus = loc["nI"] + loc["nB"]
    L = sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n_plus, 4 * nt))
    return L @ xi.reshape(4 * nt, k)


def sketch_W(mesh, s, loc, k, seed, mode, R_BB=None):
    if mode == "field":
        v = field_sketch_rhs(mesh, s, loc, k, seed)
        g = splu(loc["H_plus"].tocsc()).solve(v)
        return g[loc["nI"]:]
    if mode == "paper":
        S = node_normals(seed, s["i"], s["B"], k).astype(np.float64)
        return sla.solve_triangular(R_BB, S)
    raise ValueError(mode)


def local_basis(mesh, kappa, s, rank, oversample=0, seed=0, sketch="field",
                explicit=False, eps=None, tau=1e-12, f=None, keep_all=False,
                h1_weighted=False, rbb="auto"):
    """rbb: "always" forms R_BB (Lemma 4.1) and takes the SVD of B of Eq. (24) as
    printed; "never" (field sketch only) takes the same singular values and left
    singular vectors from B B^T = T^T S_B^{-1} T with S_B^{-1} T = ((H^+)^{-1} [0; T])_B
    (Lemma 4.1 and the block inverse of H^+), which avoids the dense Schur complement
    of large subdomains; "auto" forms R_BB where the explicit SVD or the paper's sketch
    needs it, or where H^+ is small enough for a dense Cholesky."""
    loc = local_system(mesh, kappa, s, f, h1_weighted)
    C, D = loc["C"], loc["D"]
    luA = splu(loc["A_II"])
    u0 = luA.solve(loc["b_I"])
    q0 = C @ u0
    R_i = np.linalg.cholesky(loc["H_i"].toarray()).T
    # R_BB (Lemma 4.1) enters the explicit SVD and the paper's sketch W = R_BB^{-1} S;
    # the field sketch and the two left solves of the randomized path do not need it
    need_rbb = explicit or sketch == "paper" or rbb == "always" or (
        rbb == "auto" and loc["H_plus"].shape[0] <= 6000)
    R_BB = weight_rbb(loc["H_plus"], loc["nI"]) if need_rbb else None
    out = dict(i=s["i"], nI=loc["nI"], nB=loc["nB"], n_omega=len(s["omega"]),
               owned=s["owned"], u0=u0)
    if explicit:
        Z = C @ luA.solve(loc["A_IB"].toarray())
        Yf = R_i @ sla.solve_triangular(R_BB, Z.T, trans="T").T   # R_i Z R_BB^{-1}
        U, sig, _ = np.linalg.svd(Yf, full_matrices=False)
        UU = U
    else:
        k = rank + oversample
        W = sketch_W(mesh, s, loc, k, seed, sketch, R_BB)
        Y = R_i @ (C @ luA.solve(loc["A_IB"] @ W))
        Qh, _ = np.linalg.qr(Y)
        # B = Qh^T R_i C A_II^{-1} A_IB R_BB^{-1}, right to left with k solves:
        t1 = C.T @ (R_i.T @ Qh)                    # (Qh^T R_i C)^T
        t2 = luA.solve(t1, trans="T")              # A_II^{-T} (...)
        t3 = loc["A_IB"].T @ t2                    # ((...)^T A_IB)^T
        if R_BB is not None:
            t4 = sla.solve_triangular(R_BB, t3, trans="T")  # R_BB^{-T} (...)
            Bm = t4.T
        else:
            # B B^T = t3^T S_B^{-1} t3 with S_B = R_BB^T R_BB (Lemma 4.1), and
            # S_B^{-1} t3 = ((H^+)^{-1} [0; t3])_B (block inverse of H^+): the same
            # singular values and left singular vectors as B without forming R_BB
            nI = loc["nI"]
            g = splu(loc["H_plus"].tocsc()).solve(
                np.vstack([np.zeros((nI, t3.shape[1])), t3]))[nI:]
            G = t3.T @ g
            lam, Uh = np.linalg.eigh(0.5 * (G + G.T))
            lam, Uh = lam[::-1], Uh[:, ::-1]
            sig = np.sqrt(np.maximum(lam, 0.0))
            Bm = None
        if Bm is not None:
            Uh, sig, _ = np.linalg.svd(Bm, full_matrices=False)
        UU = Qh @ Uh
        out["W"] = W
    if eps is not None:
        m = int(np.sum(sig > eps))
    elif keep_all:
        m = int(np.sum(sig > 1e-14 * sig[0]))
    else:
        m = min(rank, len(sig))
    cols = sla.solve_triangular(R_i, UU[:, :m])          # R_i^{-1} U_m
    V = D @ np.column_stack([q0, cols])
    A_PP = loc["A_PP"]
    K = V.T @ (A_PP @ V)
    lam, Wv = np.linalg.eigh(0.5 * (K + K.T))
    lam, Wv = lam[::-1], Wv[:, ::-1]
    keep = lam > tau * lam[0]
    Q = (V @ Wv[:, keep]) / np.sqrt(lam[keep])
    out.update(sigma=sig, m=m, cols=cols, q0=q0, V=V, Q=Q, lam=lam, n_kept=int(keep.sum()),
               bt=Q.T @ loc["b_P"], Kii=Q.T @ (A_PP @ Q), A_PP=A_PP, b_P=loc["b_P"],
               R_i=R_i, R_BB=R_BB)
    return out
