"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller normals.

Oracle-side implementation of the counter-based generator the solver uses
to draw its random start (Alg. 2, Step 1).  Written from the published
definition: 10 rounds of the Philox S-box on a 4x32-bit counter with a
2x32-bit key bumped by the Weyl constants between rounds.

Pinned by the Random123 known-answer vectors (tests/test_oracle_pins.py).

Normal draws: element e of an n x c column-major block in stream s uses
counter (t mod 2^32, t div 2^32, s, 0) with t = e // 2 and key (seed_lo, seed_hi); the first
two output words w0, w1 give u1 = (w0 + 0.5) / 2^32, u2 = (w1 + 0.5) / 2^32
and the pair z = sqrt(-2 ln u1) * (cos 2 pi u2, sin 2 pi u2) for elements
2t and 2t + 1.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: uint32 array (..., 4); key: uint32 array (..., 2) -> (..., 4)."""
    c = np.array(ctr, dtype=np.uint32).copy()
    k = np.array(key, dtype=np.uint32).copy()
    c0, c1, c2, c3 = (c[..., i].astype(np.uint64) for i in range(4))
    k0 = k[..., 0].astype(np.uint64)
    k1 = k[..., 1].astype(np.uint64)
    for rnd in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
        if rnd != 9:
            k0 = (k0 + np.uint64(_W0)) & _MASK
            k1 = (k1 + np.uint64(_W1)) & _MASK
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def normal_block(n: int, ncols: int, seed: int, stream: int) -> np.ndarray:
    """n x ncols float64 N(0,1) block (Fortran order) per the module rule."""
    total = n * ncols
    npair = (total + 1) // 2
    t = np.arange(npair, dtype=np.uint64)
    ctr = np.zeros((npair, 4), dtype=np.uint32)
    ctr[:, 0] = (t & _MASK).astype(np.uint32)
    ctr[:, 1] = (t >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(stream)
    key = np.zeros((npair, 2), dtype=np.uint32)
    key[:, 0] = np.uint32(seed & 0xFFFFFFFF)
    key[:, 1] = np.uint32((seed >> 32) & 0xFFFFFFFF)
    w = philox4x32_10(ctr, key)
    u1 = (w[:, 0].astype(np.float64) + 0.5) * (1.0 / 4294967296.0)
    u2 = (w[:, 1].astype(np.float64) + 0.5) * (1.0 / 4294967296.0)
    rad = np.sqrt(-2.0 * np.log(u1))
    ang = 2.0 * np.pi * u2
    z = np.empty(2 * npair)
    z[0::2] = rad * np.cos(ang)
    z[1::2] = rad * np.sin(ang)
    return np.asfortranarray(z[:total].reshape(ncols, n).T)
