"""Pins for the oracle's counter-based Gaussian generator (Sec. 6: Gaussian S_i)."""
import numpy as np
import pytest

from conftest import golden
from oracle import rng


def test_philox_known_answers():
    # published known-answer vectors of Philox-4x32-10 (Salmon et al., SC'11)
    rows = golden("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = rng.philox4x32_10(*[np.uint64(x) for x in v[:6]])
        assert [int(o) for o in out] == v[6:]


def test_uniform_is_exact_and_open():
    x = np.array([0, 1, 511, 512, 0xFFFFFFFF], dtype=np.uint32)
    u = rng.uniform01(x)
    assert u.dtype == np.float32
    expect = (2.0 * (x.astype(np.float64) // 512) + 1.0) / 2.0 ** 24
    assert np.array_equal(u.astype(np.float64), expect)
    assert u.min() > 0 and u.max() < 1


def test_ln_within_binary32_error_bound():
    u = np.random.default_rng(0).random(200000).astype(np.float32)
    u = np.clip(u, np.float32(2.0 ** -24), np.float32(1 - 2.0 ** -24))
    ref = np.log(u.astype(np.float64))
    err = np.abs(rng.ln_f32(u).astype(np.float64) - ref)
    # a few binary32 ulps of |ln u| plus one ulp of e*ln2
    assert np.all(err <= 4.0 * 2.0 ** -24 * np.abs(ref) + 2.0 ** -22)


def test_sincos_within_binary32_error_bound():
    u = ((np.arange(0, 2 ** 24, 37, dtype=np.int64) * 2 + 1) / 2.0 ** 25).astype(np.float32)
    c, s = rng.sincos_2pi_f32(u)
    a = 2.0 * np.pi * u.astype(np.float64)
    assert np.max(np.abs(c - np.cos(a))) < 3e-7
    assert np.max(np.abs(s - np.sin(a))) < 3e-7
    # octant symmetries are exact: the 8 octants reuse the same polynomial values
    assert np.allclose(c * c + s * s, 1.0, atol=1e-6)


def test_box_muller_moments():
    z = rng.field_normals(1234, 3, np.arange(50000), 4).astype(np.float64).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert abs(np.mean(z ** 3)) < 5 * np.sqrt(15.0 / n)
    assert abs(np.mean(z ** 4) - 3.0) < 5 * np.sqrt(96.0 / n)


def test_draws_depend_on_every_counter_word():
    base = rng.field_normals(7, 2, np.array([5]), 3)
    assert not np.array_equal(base, rng.field_normals(8, 2, np.array([5]), 3))
    assert not np.array_equal(base, rng.field_normals(7, 3, np.array([5]), 3))
    assert not np.array_equal(base, rng.field_normals(7, 2, np.array([6]), 3))
    assert not np.array_equal(base[:, :, 0], base[:, :, 1])
    # the field and node streams use different tags
    assert not np.array_equal(rng.node_normals(7, 2, np.array([5]), 3)[0], base[0, 0])


@pytest.mark.parametrize("seed", [0, 2 ** 40 + 17])
def test_key_uses_both_seed_words(seed):
    k0, k1 = rng.seed_key(seed)
    assert int(k0) == seed & 0xFFFFFFFF and int(k1) == seed >> 32
