"""Step 1 of the library on the host, without a GPU (mor_debug_plan_check).

- Streamed plans: every wave's rows, Morton codes, sparsity pattern, assembly
  incidences and row-space maps equal the matching rows of the one-shot plan (so a wave
  runs exactly the arithmetic of the one-shot batch on its subdomains).
- Coarse level: aggregates are contiguous runs of rows, the I aggregates precede the B
  aggregates, at most 1024 per subdomain and at most 32 meet one 128-row tile (the sizes
  the CUDA kernels are written for).
- The plan's subdomain count and owned DOFs equal the oracle's sets.
"""
import numpy as np
import pytest

import synth
from oracle import subdomains as osub


@pytest.fixture(scope="module")
def mor():
    from paper_2404_06260_gb300 import _build
    _build.build()
    from paper_2404_06260_gb300 import mor as m
    return m


@pytest.mark.parametrize("name,wave", [("cube16_p2", 3), ("cube64_p4", 10),
                                       ("cube96_kmeans", 37)])
def test_waves_equal_the_one_shot_plan_and_aggregates_fit(mor, name, wave):
    mesh, kappa, owner, p = synth.workload(name)
    c = mor.plan_check(mesh, owner, p["r_hops"], wave)
    n_sub = int(owner.max()) + 1
    assert c["n_sub"] == n_sub
    assert c["waves"] == (n_sub + wave - 1) // wave
    assert c["wave_mismatches"] == 0
    assert c["aggregate_violations"] == 0
    assert 1 <= c["max_slots"] <= 32
    assert 1 <= c["max_aggregates"] <= 1024
    assert c["owned"] == int(np.sum(mesh.dirichlet == 0))


def test_owned_sets_match_the_oracle(mor):
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    c = mor.plan_check(mesh, owner, p["r_hops"], 8)
    subs = osub.all_subdomains(mesh, owner, p["r_hops"])
    assert c["owned"] == sum(len(s["owned"]) for s in subs)
    assert c["rows"] == sum(len(s["I"]) + len(s["B"]) for s in subs)


def test_bad_partition_is_an_error_not_a_crash(mor):
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    bad = owner.copy()
    bad[bad == 3] = 9                       # label 3 unused
    with pytest.raises(mor.MorError):
        mor.plan_check(mesh, bad, p["r_hops"], 4)


def test_single_subdomain_is_rejected_with_a_clear_error(mor):
    # one subdomain: its extension is the whole domain, B is empty and Eq. (8) has no
    # boundary data; the library refuses the plan instead of building empty batches
    mesh, kappa, owner, p = synth.workload("cube16_p2")
    with pytest.raises(mor.MorError, match="empty boundary set B"):
        mor.plan_check(mesh, np.zeros_like(owner), p["r_hops"], 1)
    # two subdomains are the smallest valid partition
    two = (mesh.xyz[:, 0] > 0.5).astype(owner.dtype)
    c = mor.plan_check(mesh, two, p["r_hops"], 2)
    assert c["n_sub"] == 2 and c["wave_mismatches"] == 0


@pytest.mark.parametrize("seed", range(6))
def test_random_partitions_match_the_oracle(mor, seed):
    # seeded k-means partitions of a jittered 10^3 cube, random hops and wave size:
    # either every invariant holds, or (an extension covering the domain) the plan is
    # rejected exactly when the oracle finds a subdomain with an empty B
    rng = np.random.default_rng(100 + seed)
    mesh = synth.kuhn_cube(10, jitter=0.2, seed=200 + seed)
    parts = int(rng.integers(3, 9))
    owner = synth.kmeans_owner(mesh, parts, 300 + seed)
    r_hops = int(rng.integers(1, 5))
    n_sub = int(owner.max()) + 1
    wave = int(rng.integers(1, n_sub + 1))
    subs = osub.all_subdomains(mesh, owner, r_hops)
    if any(len(s["B"]) == 0 for s in subs):
        with pytest.raises(mor.MorError, match="empty boundary set B"):
            mor.plan_check(mesh, owner, r_hops, wave)
        return
    c = mor.plan_check(mesh, owner, r_hops, wave)
    assert c["n_sub"] == n_sub and c["wave_mismatches"] == 0
    assert c["aggregate_violations"] == 0
    assert c["owned"] == sum(len(s["owned"]) for s in subs)
    assert c["rows"] == sum(len(s["I"]) + len(s["B"]) for s in subs)


def test_finer_aggregates_pass_the_old_cap(mor):
    # coarse_rows 35 (the mixed default) on the 64^3 workload: the interior subdomains take
    # more than 256 aggregates (the A_II and H^+ sets of the coarse level), still within
    # the caps
    mesh, kappa, owner, p = synth.workload("cube64_p4")
    c = mor.plan_check(mesh, owner, p["r_hops"], 64, coarse_rows=35)
    assert c["aggregate_violations"] == 0
    assert 256 < c["max_aggregates"] <= 1024
    assert 1 <= c["max_slots"] <= 32
