"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11), FP64 oracle side.

Written from the published definition: a 4x32-bit counter is passed through ten
rounds; each round multiplies words 0 and 2 by the constants 0xD2511F53 and
0xCD9E8D57, splits the 64-bit products into high and low halves, xors the high
halves with the other counter words and the round key, and permutes; the 2x32
key is bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds.

The stream layout of the sampler (the paper draws its Monte Carlo samples on the
CPU, Sec. II.B; here both sides draw the same bits): key = (seed low 32, seed
high 32); counter = (sample index, round, block, point).  Block b of sample i
supplies uniforms 4b..4b+3 of that sample.
"""
from __future__ import annotations

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: (4, ...) integers < 2^32; key: (2, ...) integers < 2^32. Returns (4, ...) uint32."""
    c = [np.asarray(x, dtype=np.uint64) & _MASK for x in ctr]
    k0 = np.asarray(key[0], dtype=np.uint64) & _MASK
    k1 = np.asarray(key[1], dtype=np.uint64) & _MASK
    for r in range(10):
        if r:
            k0 = (k0 + np.uint64(_W0)) & _MASK
            k1 = (k1 + np.uint64(_W1)) & _MASK
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack([x.astype(np.uint32) for x in c])


def bits_to_uniform(x):
    """u = (floor(x / 2^9) + 1/2) / 2^23, in (0, 1); exactly representable in float32."""
    x = np.asarray(x, dtype=np.uint64)
    return ((x >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def uniforms(seed: int, point: int, rnd: int, idx, n_dims: int):
    """Uniforms (n_dims, len(idx)) for samples idx of one (point, round)."""
    idx = np.asarray(idx, dtype=np.uint64)
    key = (np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))
    out = np.empty((n_dims, idx.shape[0]))
    for b in range((n_dims + 3) // 4):
        ctr = (idx, np.full_like(idx, rnd), np.full_like(idx, b), np.full_like(idx, point))
        bits = philox4x32_10(ctr, key)
        for j in range(4):
            d = 4 * b + j
            if d < n_dims:
                out[d] = bits_to_uniform(bits[j])
    return out
