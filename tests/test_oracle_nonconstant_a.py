"""The paper's nonconstant-coefficient test (Sec. 7.3) with the oracle.

The paper takes a(x) = 10^k sin(100 x) + 10^k + 1, k = 1, 2, 3, on its case-5 mesh
(30481 DOFs, 30 subdomains), 6 hops, eps = 1e-2 and explicit weighted SVDs, and prints
reduction errors of 6.5e-5, 2.0e-5 and 6.3e-6 (tests/golden/sec73_nonconstant_a.txt).
Each step divides the error by 3.25 and 3.17, i.e. by about sqrt(10): these are errors
in the energy norm of a, which scales like a^(-1/2) when the relative error does not
depend on k.

That mesh (unstructured, METIS-partitioned) is not available.  A 24^3 Kuhn cube
(12,167 DOFs, h = 0.072 against the paper's 0.099) with 30 seeded k-means subdomains
stands in, with the paper's load f (Sec. 7.1).  The pins are:
- the relative reduction error does not depend on k (within 10%);
- the absolute energy-norm error falls by 2.5..3.8 per step of k (paper: 3.25, 3.17);
- its size is that of the paper's at every k, within a factor of 5 (mesh and
  partition differ; measured: 2.9x at all three k).
"""
import numpy as np
import pytest

import synth
from conftest import golden
from oracle import pipeline, reduced


def _paper_load(x, y, z):
    return 60.0 * ((1 - x) * x * (1 - y) * y + (1 - x) * x * (1 - z) * z +
                   (1 - y) * y * (1 - z) * z)


@pytest.fixture(scope="module")
def runs():
    mesh = synth.kuhn_cube(24)
    owner = synth.kmeans_owner(mesh, 30, 1005)
    out = {}
    for k in (1, 2, 3):
        a = synth.sine_kappa(mesh, k)
        r = pipeline.run(mesh, a, owner, rank=0, oversample=0, r_hops=6, seed=1005,
                         explicit=True, eps=1e-2, f=_paper_load)
        out[k] = (r["red_err"], reduced.energy_norm(mesh, a, r["u"] - r["u_red"]))
    return out


def test_coefficient_contrast_matches_the_paper():
    mesh = synth.kuhn_cube(24)
    a = synth.sine_kappa(mesh, 3)
    assert 1500 < a.max() / a.min() <= 2001          # "2001 : 1" for k = 3


def test_relative_reduction_error_does_not_depend_on_k(runs):
    rel = [runs[k][0] for k in (1, 2, 3)]
    assert max(rel) < 1.1 * min(rel)
    assert max(rel) < 1e-3                           # eps = 1e-2 gives O(1e-4), Table 1


def test_absolute_error_trend_and_size_match_the_paper(runs):
    paper = {int(r[0]): float(r[1]) for r in golden("sec73_nonconstant_a.txt")}
    for k in (1, 2):
        ratio = runs[k][1] / runs[k + 1][1]
        assert 2.5 < ratio < 3.8, (k, ratio)
        assert 2.5 < paper[k] / paper[k + 1] < 3.8
    for k in (1, 2, 3):
        assert paper[k] / 5 < runs[k][1] < paper[k] * 5, (k, runs[k][1], paper[k])
