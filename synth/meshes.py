"""Seeded mesh, coefficient and partition generators.

Mesh: the unit cube split into n^3 hexahedral cells, each cut into the six tetrahedra
of the Kuhn (Freudenthal) subdivision 0 -> e_p1 -> e_p1+e_p2 -> (1,1,1) over the six
permutations p of the axes, with the same orientation in every cell so the mesh is
conforming.  This is the structured tetrahedral cube of the paper's scaling tests
(Sec. 7.1: dim V = (n-1)^3 interior nodes, h = sqrt(3)/n, cases 7-11).

Every tetrahedron is stored with positive orientation (det[v1-v0, v2-v0, v3-v0] > 0).
Dirichlet nodes are those on the cube's surface (u = 0 on the boundary, Eq. (1)).
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

# the six axis permutations, in lexicographic order
_PERMS = list(itertools.permutations(range(3)))


@dataclasses.dataclass
class Mesh:
    n: int                 # cells per side
    xyz: np.ndarray        # (n_nodes, 3) float64
    tets: np.ndarray       # (n_tets, 4) int32, positively oriented
    dirichlet: np.ndarray  # (n_nodes,) uint8, 1 on the cube surface

    @property
    def n_nodes(self) -> int:
        return self.xyz.shape[0]

    @property
    def n_tets(self) -> int:
        return self.tets.shape[0]


def node_id(ix, iy, iz, n):
    """Lexicographic node numbering, x fastest."""
    return ix + (n + 1) * (iy + (n + 1) * iz)


def kuhn_cube(n: int, jitter: float = 0.0, seed: int = 0) -> Mesh:
    """Structured n^3-cell unit cube, 6 Kuhn tetrahedra per cell.

    jitter > 0 moves every interior node by U(-jitter*h, jitter*h) per coordinate
    (seeded); the seed is rejected (ValueError) if any tetrahedron would invert.
    Without jitter every cell is a translate of the first, so each of the 6 Kuhn
    permutations is oriented once (int32 arrays throughout: the 440^3 cube has 5.1e8
    tetrahedra).
    """
    h = 1.0 / n
    g = np.arange(n + 1, dtype=np.float64) * h
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    del x, y, z

    c = np.arange(n, dtype=np.int32)
    cz, cy, cx = np.meshgrid(c, c, c, indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()
    tets = np.empty((n ** 3, 6, 4), dtype=np.int32)
    for p, perm in enumerate(_PERMS):
        off = np.zeros((4, 3), dtype=np.int32)
        off[1, perm[0]] = 1
        off[2] = off[1]
        off[2, perm[1]] += 1
        off[3] = 1
        col = [0, 1, 2, 3]
        if jitter == 0.0 and np.linalg.det((off[1:] - off[0]).astype(np.float64)) < 0:
            col = [0, 2, 1, 3]          # positive orientation: swap vertices 1 and 2
        for a in range(4):
            tets[:, p, col[a]] = node_id(cx + off[a, 0], cy + off[a, 1], cz + off[a, 2], n)
    del cx, cy, cz
    tets = tets.reshape(-1, 4)

    ii = np.arange(n + 1)
    on_face = (ii == 0) | (ii == n)
    fz, fy, fx = np.meshgrid(on_face, on_face, on_face, indexing="ij")
    dirichlet = (fx | fy | fz).ravel().astype(np.uint8)

    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
        d[dirichlet.astype(bool)] = 0.0
        xyz = xyz + d
        # orient every tetrahedron positively, then reject inverted ones
        e = xyz[tets[:, 1:]] - xyz[tets[:, :1]]
        det = np.einsum("ti,ti->t", e[:, 0], np.cross(e[:, 1], e[:, 2]))
        neg = det < 0
        tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
        e = xyz[tets[:, 1:]] - xyz[tets[:, :1]]
        det = np.einsum("ti,ti->t", e[:, 0], np.cross(e[:, 1], e[:, 2]))
        if np.any(det <= 0):
            raise ValueError("jitter seed inverts a tetrahedron; choose another seed")
    return Mesh(n=n, xyz=np.ascontiguousarray(xyz), tets=np.ascontiguousarray(tets),
                dirichlet=dirichlet)


def kuhn_box_tets(n: int, lo, hi) -> np.ndarray:
    """Ids of the tetrahedra of kuhn_cube(n) in the cells lo <= (cx, cy, cz) < hi
    (clipped to the cube): cell (cx, cy, cz) holds tetrahedra 6 c .. 6 c + 5 with
    c = cx + n (cy + n cz)."""
    lo = [max(0, int(v)) for v in lo]
    hi = [min(n, int(v)) for v in hi]
    cz, cy, cx = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]),
                             np.arange(lo[0], hi[0]), indexing="ij")
    c = (cx + n * (cy + n * cz)).ravel().astype(np.int64)
    return (6 * c[:, None] + np.arange(6)[None, :]).ravel()


def box_node_range(n: int, parts: int, a: int):
    """Node index range [lo, hi) along one axis owned by box a of box_owner(n, parts)."""
    i = np.arange(n + 1)
    own = np.flatnonzero(np.minimum(parts - 1, (i * parts) // n) == a)
    return int(own[0]), int(own[-1]) + 1


def lognormal_kappa(n_tets: int, seed: int) -> np.ndarray:
    """k_T = exp(g_T), g_T iid N(0,1) per element."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.standard_normal(n_tets))


def sine_kappa(mesh: Mesh, k: int) -> np.ndarray:
    """The oscillating coefficient of the paper's nonconstant-a test (Sec. 7.3),
    a(x) = 10^k sin(100 x) + 10^k + 1, evaluated at the element centroids (a P0 field);
    max/min over the cube approaches 2001 for k = 3."""
    x = mesh.xyz[mesh.tets][:, :, 0].mean(axis=1)
    return 10.0 ** k * np.sin(100.0 * x) + 10.0 ** k + 1.0


def sphere_kappa(mesh: Mesh, seed: int, contrast: float = 1e4, fill: float = 0.10,
                 rmin_h: float = 3.0, rmax_h: float = 6.0) -> np.ndarray:
    """k = 1 background, k = contrast inside seeded random spheres of radius
    U[rmin_h*h, rmax_h*h], spheres added until >= fill of the elements have their
    centroid inside one."""
    rng = np.random.default_rng(seed)
    h = 1.0 / mesh.n
    cen = mesh.xyz[mesh.tets].mean(axis=1)
    inside = np.zeros(mesh.n_tets, dtype=bool)
    while inside.mean() < fill:
        c = rng.uniform(0.0, 1.0, size=3)
        r = rng.uniform(rmin_h * h, rmax_h * h)
        inside |= np.sum((cen - c) ** 2, axis=1) < r * r
    k = np.ones(mesh.n_tets)
    k[inside] = contrast
    return k


def box_owner(n: int, parts: int) -> np.ndarray:
    """Box partition of the (n+1)^3 nodes into parts^3 owner labels:
    owner_axis = min(parts-1, floor(i*parts/n))."""
    i = np.arange(n + 1)
    a = np.minimum(parts - 1, (i * parts) // n)
    az, ay, ax = np.meshgrid(a, a, a, indexing="ij")
    return (ax + parts * (ay + parts * az)).ravel().astype(np.int32)


def slab_owner(n: int, parts: int, axis: int = 0) -> np.ndarray:
    """Owner labels by slabs along one axis: floor(i*parts/n) clipped to parts-1."""
    i = np.arange(n + 1)
    a = np.minimum(parts - 1, (i * parts) // n)
    az, ay, ax = np.meshgrid(a, a, a, indexing="ij")
    return [ax, ay, az][axis].ravel().astype(np.int32)


def kmeans_owner(mesh: Mesh, parts: int, seed: int, iters: int = 20,
                 sample: int = 200000) -> np.ndarray:
    """Owner labels from k-means on element centroids: Lloyd iterations (seeded
    k-means++ start) on a seeded sample of `sample` centroids, then every node is owned
    by its nearest centre.  Labels are renumbered 0..n-1 over the centres that own a
    node."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    cen = mesh.xyz[mesh.tets].mean(axis=1)
    pts = cen[rng.choice(len(cen), size=min(sample, len(cen)), replace=False)]
    C = np.empty((parts, 3))
    C[0] = pts[rng.integers(len(pts))]
    d2 = np.sum((pts - C[0]) ** 2, axis=1)
    for j in range(1, parts):
        C[j] = pts[rng.choice(len(pts), p=d2 / d2.sum())]
        d2 = np.minimum(d2, np.sum((pts - C[j]) ** 2, axis=1))
    for _ in range(iters):
        lab = cKDTree(C).query(pts)[1]
        cnt = np.bincount(lab, minlength=parts)
        for ax in range(3):
            sums = np.bincount(lab, weights=pts[:, ax], minlength=parts)
            C[cnt > 0, ax] = sums[cnt > 0] / cnt[cnt > 0]
    owner = cKDTree(C).query(mesh.xyz)[1]
    _, owner = np.unique(owner, return_inverse=True)
    return owner.astype(np.int32)


# Workloads (sizes of the paper's structured scaling meshes, Sec. 7.1, scaled down
# for the small cases).  rank = kept singular vectors, oversample = extra sketch
# columns, r_hops = extension hops (about half the subdomain width, so the extension
# roughly doubles the subdomain diameter), mixed_rtol = local-solve tolerance of the
# mixed-precision path where the default 1e-9 is too loose for 1e-6 in energy.
WORKLOADS = {
    "cube16_p2": dict(n=16, parts=2, rank=8, oversample=5, r_hops=4, field="lognormal",
                      seed=1001),
    "cube64_p4": dict(n=64, parts=4, rank=32, oversample=10, r_hops=8, field="lognormal",
                      seed=1002),
    "cube96_kmeans": dict(n=96, parts=300, rank=0, oversample=10, r_hops=-1,
                          field="lognormal", seed=1003, jitter=0.2, partition="kmeans",
                          rank_range=(16, 64)),
    "cube128_p8_spheres": dict(n=128, parts=8, rank=48, oversample=10, r_hops=8,
                               field="spheres", seed=1004, mixed_rtol=1e-11),
    "cube440_p20": dict(n=440, parts=20, rank=32, oversample=10, r_hops=11,
                        field="lognormal", seed=1005),
}


def workload(name: str, **override):
    """Return (mesh, kappa, owner, params) for a named workload.  For workloads with a
    rank range, params["ranks"] holds the seeded per-subdomain ranks (uniform in the
    range, inclusive) and params["r_hops"] = -1 selects the per-subdomain hop rule
    max(1, round(|P_i|^(1/3) / 2))."""
    p = dict(WORKLOADS[name])
    p.update(override)
    mesh = kuhn_cube(p["n"], jitter=p.get("jitter", 0.0), seed=p["seed"])
    if p["field"] == "lognormal":
        kappa = lognormal_kappa(mesh.n_tets, p["seed"])
    elif p["field"] == "ones":
        kappa = np.ones(mesh.n_tets)
    else:
        kappa = sphere_kappa(mesh, p["seed"])
    if p.get("partition") == "kmeans":
        owner = kmeans_owner(mesh, p["parts"], p["seed"])
    else:
        owner = box_owner(p["n"], p["parts"])
    if "rank_range" in p:
        lo, hi = p["rank_range"]
        n_sub = int(owner.max()) + 1
        p["ranks"] = np.random.default_rng(p["seed"] + 7).integers(lo, hi + 1, size=n_sub)
    return mesh, kappa, owner, p
