"""Pins for the oracle's overlapping subdomains and r-hop extensions (Sec. 3, Sec. 7.1),
checked against brute-force Python definitions on tiny meshes."""
from collections import deque

import numpy as np

import synth
from oracle import subdomains as sd


def _brute_sets(mesh, owner, i, r):
    nbr = [set() for _ in range(mesh.n_nodes)]
    inc = [[] for _ in range(mesh.n_nodes)]
    for t, tet in enumerate(mesh.tets.tolist()):
        for a in tet:
            inc[a].append(t)
            nbr[a].update(tet)
    dist = {v: 0 for v in range(mesh.n_nodes) if owner[v] == i}
    q = deque(dist)
    while q:
        v = q.popleft()
        if dist[v] == r:
            continue
        for w in nbr[v]:
            if w not in dist:
                dist[w] = dist[v] + 1
                q.append(w)
    plus = {t for t, tet in enumerate(mesh.tets.tolist()) if any(a in dist for a in tet)}
    nodes = {a for t in plus for a in mesh.tets[t].tolist()}
    free = lambda v: mesh.dirichlet[v] == 0
    I = sorted(v for v in nodes if free(v) and all(t in plus for t in inc[v]))
    B = sorted(v for v in nodes if free(v) and v not in set(I))
    omega_t = {t for t, tet in enumerate(mesh.tets.tolist()) if any(owner[a] == i for a in tet)}
    omega = sorted({a for t in omega_t for a in mesh.tets[t].tolist() if free(a)})
    return I, B, omega, sorted(plus), sorted(omega_t)


def test_sets_match_brute_force():
    mesh = synth.kuhn_cube(6, jitter=0.2, seed=11)
    owner = synth.box_owner(6, 2)
    for i in (0, 5):
        for r in (1, 2):
            s = sd.subdomain_sets(mesh, owner, i, r)
            I, B, omega, plus, omega_t = _brute_sets(mesh, owner, i, r)
            assert s["I"].tolist() == I
            assert s["B"].tolist() == B
            assert s["omega"].tolist() == omega
            assert s["plus_tets"].tolist() == plus
            assert s["omega_tets"].tolist() == omega_t


def test_owned_nodes_partition_the_free_nodes():
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    subs = sd.all_subdomains(mesh, owner, p["r_hops"])
    cnt = np.zeros(mesh.n_nodes, dtype=int)
    for s in subs:
        cnt[s["owned"]] += 1
        assert np.intersect1d(s["I"], s["B"]).size == 0
        assert np.all(np.isin(s["omega"], s["I"]))
        assert np.all(np.isin(s["owned"], s["omega"]))
    assert np.array_equal(cnt, (mesh.dirichlet == 0).astype(int))


def test_overlap_is_one_element_layer():
    # two subdomains omega_i, omega_j meet in one layer of elements (Sec. 3):
    # every shared element has vertices owned by both
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    subs = sd.all_subdomains(mesh, owner, p["r_hops"])
    t0 = sd.interface_tets(mesh, owner)
    cover = np.zeros(mesh.n_tets, dtype=int)
    for s in subs:
        cover[s["omega_tets"]] += 1
    assert np.array_equal(np.flatnonzero(cover >= 2), t0)
    assert cover.min() == 1


def test_region_sets_equal_whole_mesh_sets():
    # the restricted computation (for meshes too large for a global adjacency) gives
    # the sets of the whole-mesh computation when its candidate elements reach r + 2
    # cells beyond the owned box; with too small a region it must not silently agree
    n, parts, r = 24, 3, 4
    mesh = synth.kuhn_cube(n)
    owner = synth.box_owner(n, parts)
    adj = sd.node_adjacency(mesh.tets, mesh.n_nodes)
    for i in (0, 4, 13, 26):
        a = (i % parts, (i // parts) % parts, i // parts ** 2)
        rng = [synth.box_node_range(n, parts, v) for v in a]
        lo = [x[0] - r - 2 for x in rng]
        hi = [x[1] + r + 1 for x in rng]
        reg = synth.kuhn_box_tets(n, lo, hi)
        got = sd.subdomain_sets_region(mesh, owner, i, r, reg)
        ref = sd.subdomain_sets(mesh, owner, i, r, adj)
        for key in ("I", "B", "omega", "owned", "plus_tets", "omega_tets"):
            assert np.array_equal(got[key], ref[key]), (i, key)
    # a region one hop short misclassifies boundary nodes of the extension
    i = 13
    rng = [synth.box_node_range(n, parts, 1) for _ in range(3)]
    reg = synth.kuhn_box_tets(n, [x[0] - r + 1 for x in rng], [x[1] + r - 1 for x in rng])
    got = sd.subdomain_sets_region(mesh, owner, i, r, reg)
    ref = sd.subdomain_sets(mesh, owner, i, r, adj)
    assert not np.array_equal(got["B"], ref["B"])
