"""Counter-based Gaussian draws for the sketch (Sec. 6, "Randomized numerical linear
algebra": the standard Gaussian test matrix S_i).

Generator: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC'11): a 4x32-bit counter and 2x32-bit key, ten rounds of
  (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2,
  c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
with the key bumped by the Weyl constants (W0, W1) between rounds.

Normals: Box-Muller (Box & Muller 1958), z0 = r cos(2 pi u2), z1 = r sin(2 pi u2),
r = sqrt(-2 ln u1), evaluated in IEEE binary32 with a FIXED sequence of correctly
rounded operations (+, -, *, /, sqrt only, no fused multiply-add):
  ln u     = e ln2 + 2 s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9),  s = (m-1)/(m+1),
             u = m 2^e with m in [sqrt(2)/2, sqrt(2)]  (atanh series),
  sin, cos = Taylor polynomials of degree 9 / 10 on [0, pi/4] after an exact octant
             reduction of u2.
Because every step is a correctly rounded binary32 operation, any implementation of
this sequence draws bit-identical normals; the truncation errors (< 1e-9) are far
below binary32 rounding.

Draw layout used by the method:
  field sketch   xi_T[a, j], a = 0..3  <- Philox(ctr = (T, j, i, 0), key = seed)
  paper sketch   S[b, j]               <- first normal of Philox(ctr = (b, j, i, 1), key)
with T the global element id, b the global node id, j the column, i the subdomain.
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox-4x32 with 10 rounds on arrays of uint32 counters; returns 4 uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(c.astype(np.uint32) for c in (c0, c1, c2, c3))


_F = np.float32
# binary32 constants, written as exact hexadecimal values of the nearest binary32
_LN2 = _F(float.fromhex("0x1.62e430p-1"))
_SQRT2 = _F(float.fromhex("0x1.6a09e6p+0"))
_PI4 = _F(float.fromhex("0x1.921fb6p-1"))
_L3 = _F(float.fromhex("0x1.555556p-2"))    # 1/3
_L5 = _F(float.fromhex("0x1.99999ap-3"))    # 1/5
_L7 = _F(float.fromhex("0x1.24924ap-3"))    # 1/7
_L9 = _F(float.fromhex("0x1.c71c72p-4"))    # 1/9
_S3 = _F(float.fromhex("-0x1.555556p-3"))   # -1/3!
_S5 = _F(float.fromhex("0x1.111112p-7"))    # 1/5!
_S7 = _F(float.fromhex("-0x1.a01a02p-13"))  # -1/7!
_S9 = _F(float.fromhex("0x1.71de3ap-19"))   # 1/9!
_C2 = _F(-0.5)                              # -1/2!
_C4 = _F(float.fromhex("0x1.555556p-5"))    # 1/4!
_C6 = _F(float.fromhex("-0x1.6c16c2p-10"))  # -1/6!
_C8 = _F(float.fromhex("0x1.a01a02p-16"))   # 1/8!
_C10 = _F(float.fromhex("-0x1.27e4fcp-22"))  # -1/10!


def uniform01(x):
    """uint32 -> binary32 in (0, 1): (2*(x >> 9) + 1) * 2^-24, exact."""
    x = np.asarray(x, dtype=np.uint32)
    return ((x >> np.uint32(9)) * np.uint32(2) + np.uint32(1)).astype(np.float32) * _F(2.0 ** -24)


def ln_f32(u):
    """Natural log of binary32 u in (0, 1] by the fixed operation sequence above."""
    u = np.asarray(u, dtype=np.float32)
    bits = u.view(np.uint32)
    e = ((bits >> np.uint32(23)) & np.uint32(0xFF)).astype(np.int32) - 127
    m = ((bits & np.uint32(0x7FFFFF)) | np.uint32(0x3F800000)).view(np.float32)
    big = m > _SQRT2
    m = np.where(big, m * _F(0.5), m).astype(np.float32)
    e = e + big.astype(np.int32)
    s = (m - _F(1.0)) / (m + _F(1.0))
    s2 = s * s
    p = _L9
    p = p * s2 + _L7
    p = p * s2 + _L5
    p = p * s2 + _L3
    p = p * s2 + _F(1.0)
    lnm = (s + s) * p
    return e.astype(np.float32) * _LN2 + lnm


def sincos_2pi_f32(u):
    """(cos 2 pi u, sin 2 pi u) for binary32 u in (0, 1), fixed operation sequence."""
    u = np.asarray(u, dtype=np.float32)
    t = u * _F(8.0)                       # exact
    q = np.floor(t).astype(np.float32)    # exact
    f = t - q                             # exact
    qi = q.astype(np.int32)
    odd = (qi & 1) == 1
    g = np.where(odd, _F(1.0) - f, f).astype(np.float32)
    th = g * _PI4
    th2 = th * th
    sp = _S9
    sp = sp * th2 + _S7
    sp = sp * th2 + _S5
    sp = sp * th2 + _S3
    sp = sp * th2
    sn = th + th * sp
    cp = _C10
    cp = cp * th2 + _C8
    cp = cp * th2 + _C6
    cp = cp * th2 + _C4
    cp = cp * th2 + _C2
    cs = cp * th2 + _F(1.0)
    swap = (qi == 1) | (qi == 2) | (qi == 5) | (qi == 6)
    c = np.where(swap, sn, cs)
    s = np.where(swap, cs, sn)
    c = np.where((qi >= 2) & (qi <= 5), -c, c)
    s = np.where(qi >= 4, -s, s)
    return c.astype(np.float32), s.astype(np.float32)


def box_muller_f32(x_u1, x_u2):
    """Two uint32 draws -> two binary32 standard normals."""
    u1 = uniform01(x_u1)
    u2 = uniform01(x_u2)
    r = np.sqrt(_F(-2.0) * ln_f32(u1))
    c, s = sincos_2pi_f32(u2)
    return r * c, r * s


def seed_key(seed: int):
    return np.uint32(seed & 0xFFFFFFFF), np.uint32((seed >> 32) & 0xFFFFFFFF)


def field_normals(seed: int, sub: int, tets_global, cols):
    """xi[t, a, j] for element ids tets_global (n_t,), columns 0..cols-1: (n_t, 4, cols)
    binary32 normals, counter (T, j, sub, 0)."""
    k0, k1 = seed_key(seed)
    T = np.asarray(tets_global, dtype=np.uint64)[:, None]
    J = np.arange(cols, dtype=np.uint64)[None, :]
    T, J = np.broadcast_arrays(T, J)
    x0, x1, x2, x3 = philox4x32_10(T, J, np.full(T.shape, sub, np.uint64),
                                   np.zeros(T.shape, np.uint64), k0, k1)
    z0, z1 = box_muller_f32(x0, x1)
    z2, z3 = box_muller_f32(x2, x3)
    return np.stack([z0, z1, z2, z3], axis=1)


def node_normals(seed: int, sub: int, nodes_global, cols):
    """S[b, j] for global node ids (n_b,), columns 0..cols-1: (n_b, cols) binary32
    normals, counter (b, j, sub, 1), first normal of each draw."""
    k0, k1 = seed_key(seed)
    Bn = np.asarray(nodes_global, dtype=np.uint64)[:, None]
    J = np.arange(cols, dtype=np.uint64)[None, :]
    Bn, J = np.broadcast_arrays(Bn, J)
    x0, x1, _, _ = philox4x32_10(Bn, J, np.full(Bn.shape, sub, np.uint64),
                                 np.ones(Bn.shape, np.uint64), k0, k1)
    z0, _ = box_muller_f32(x0, x1)
    return z0
