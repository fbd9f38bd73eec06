"""Gaussian-embedding sketch, the comparator of Sec. 4 of the paper, plain
FP64 numpy. TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper validates the block SRHT against Gaussian embeddings (Sec. 4:
same approximation quality, block SRHT up to 2.5x faster to apply) and
names Gaussian matrices among the classical oblivious subspace embeddings
(Sec. 1). Definition followed: Omega_G (l x n) with independent N(0, 1/l)
entries, so that E[Omega_G^T Omega_G] = I like the block SRHT; the sketch is
B = Omega_G A for the tall n x m A.

The entries come from a counter-based generator so that any device can
reproduce them (the paper only says the local matrices come from a seeded
generator): Philox4x64-10 (``oracle.philox``) with key (seed, 0) and
counter (k >> 1, j, 3, 0) gives four 64-bit words for the pair of columns
(2 (k >> 1), 2 (k >> 1) + 1) of row j; column k uses words (0, 1) when k is
even and (2, 3) when k is odd. A word w becomes the uniform
u = (2 (w >> 41) + 1) 2^-24 in (0, 1) (exactly representable in FP32 and
FP64), and the Box-Muller transform (Box and Muller, 1958) of the pair
(u1, u2) gives z = sqrt(-2 ln u1) cos(2 pi u2) ~ N(0, 1); the entry is
z / sqrt(l).

Parity: pinned by the tests against numpy's own Philox (through the scalar
generator), the normal distribution (moments, Kolmogorov-Smirnov),
E[Omega^T Omega] = I and the Marchenko-Pastur edges of the embedding.
"""

from __future__ import annotations

import numpy as np

from .philox import MASK64, PHILOX_M0, PHILOX_M1, PHILOX_W0, PHILOX_W1, philox4x64_10

STREAM_G = 3
_M32 = np.uint64(0xFFFFFFFF)


def _mulhilo(a: np.ndarray, b: int):
    """(hi, lo) 64-bit halves of the 128-bit products a * b (uint64 arrays),
    from 32-bit limbs so that every partial product fits in 64 bits."""
    b_lo = np.uint64(b & 0xFFFFFFFF)
    b_hi = np.uint64(b >> 32)
    a_lo = a & _M32
    a_hi = a >> np.uint64(32)
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    t = (ll >> np.uint64(32)) + (lh & _M32) + (hl & _M32)
    lo = (ll & _M32) | (t << np.uint64(32))
    hi = hh + (lh >> np.uint64(32)) + (hl >> np.uint64(32)) + (t >> np.uint64(32))
    return hi, lo


def philox4x64_10_vec(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x64-10 on arrays of counters (the round function of
    ``oracle.philox.philox4x64_10``, one array lane per counter)."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64).copy() for c in (c0, c1, c2, c3))
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd:
                k0 = (k0 + PHILOX_W0) & MASK64
                k1 = (k1 + PHILOX_W1) & MASK64
            hi0, lo0 = _mulhilo(c0, PHILOX_M0)
            hi1, lo1 = _mulhilo(c2, PHILOX_M1)
            c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
    return c0, c1, c2, c3


def uniform_from_word(w: np.ndarray) -> np.ndarray:
    """u = (2 (w >> 41) + 1) 2^-24, in (0, 1), FP64 (exact)."""
    return ((np.asarray(w, dtype=np.uint64) >> np.uint64(41)).astype(np.float64) * 2.0 + 1.0) * 2.0 ** -24


def box_muller(u1: np.ndarray, u2: np.ndarray) -> np.ndarray:
    """z = sqrt(-2 ln u1) cos(2 pi u2) (Box and Muller, 1958)."""
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def omega_gaussian(n: int, l: int, seed: int) -> np.ndarray:
    """The l x n Gaussian embedding, entries N(0, 1/l) (module docstring)."""
    npair = (n + 1) // 2
    q = np.tile(np.arange(npair, dtype=np.uint64), l)
    j = np.repeat(np.arange(l, dtype=np.uint64), npair)
    w0, w1, w2, w3 = philox4x64_10_vec(q, j, np.full_like(q, STREAM_G), np.zeros_like(q), seed & MASK64, 0)
    even = box_muller(uniform_from_word(w0), uniform_from_word(w1)).reshape(l, npair)
    odd = box_muller(uniform_from_word(w2), uniform_from_word(w3)).reshape(l, npair)
    om = np.empty((l, 2 * npair), dtype=np.float64)
    om[:, 0::2] = even
    om[:, 1::2] = odd
    return om[:, :n] / np.sqrt(l)


def omega_gaussian_entry(j: int, k: int, l: int, seed: int) -> float:
    """One entry from the scalar generator (independent of the vectorised
    path; used by the tests to pin it)."""
    w = philox4x64_10((k >> 1, j, STREAM_G, 0), (seed, 0))
    a, b = (w[0], w[1]) if k % 2 == 0 else (w[2], w[3])
    u1 = ((a >> 41) * 2 + 1) * 2.0 ** -24
    u2 = ((b >> 41) * 2 + 1) * 2.0 ** -24
    return float(np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2) / np.sqrt(l))


def gaussian_sketch(a: np.ndarray, l: int, seed: int, row_panel: int = 1 << 14) -> np.ndarray:
    """B = Omega_G A (l x m), FP64; Omega_G formed in row panels of A."""
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[0]
    om = omega_gaussian(n, l, seed)
    out = np.zeros((l, a.shape[1]), dtype=np.float64)
    for k0 in range(0, n, row_panel):
        out += om[:, k0:k0 + row_panel] @ a[k0:k0 + row_panel]
    return out
