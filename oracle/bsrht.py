"""Block SRHT sketch, plain FP64 CPU restatement of Sec. 2 of the paper.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Definitions followed (orientation used throughout: A is n x m, tall; the
sketch is B = Omega A with Omega l x n):

* eq. 2.3: Omega = [Omega^(1) ... Omega^(p)],
  Omega^(i) = sqrt(r/l) * Dt^(i) R H D^(i), with one sampling matrix R shared
  by all blocks, D^(i) (r x r) and Dt^(i) (l x l) Rademacher diagonals, and H
  the r x r Walsh-Hadamard matrix scaled by 1/sqrt(r) (Sec. 2 normalises H by
  the square root of its size; the proof of Thm 2.1 uses the same 1/sqrt(r)).
  Every entry of Omega is therefore +-1/sqrt(l).
* Sec. 2 (paragraph after eq. 2.4): R samples uniformly *with replacement*.
* Sec. 2 (partial SRHT): r a power of two by zero padding. Reading used here:
  block i holds rows [i*rb, min(n, (i+1)*rb)) with rb = ceil(n/p), and r is
  the next power of two >= rb; the missing rows are zero.
* Sec. 2 (tensor form): H = (1/sqrt(r)) H2 x H2 x ... x H2 with
  H2 = [[1, 1], [1, -1]]; built here by the Sylvester recursion
  H_{2k} = [[H_k, H_k], [H_k, -H_k]] (natural, not sequency, order).
* eq. 2.4: Omega V = sum_i Omega^(i) V^(i).

The random signs and samples come from Philox4x64-10 with key (seed, 0)
(the paper only says the local matrices come from a seeded generator):

* D^(i) sign of local row k:  counter (k >> 8, i, 0, 0), output word
  (k >> 6) & 3, bit k & 63; a set bit means -1.
* Dt^(i) sign of sketch row j: counter (j >> 8, i, 1, 0), same bit rule.
* R sample s_j of sketch row j: counter (j >> 2, 0, 2, 0), output word
  j & 3, s_j = word mod r (r is a power of two, so this is unbiased).
"""

from __future__ import annotations

import functools
import math

import numpy as np

from .philox import philox4x64_10

STREAM_D = 0
STREAM_DT = 1
STREAM_R = 2


def next_pow2(x: int) -> int:
    r = 1
    while r < x:
        r <<= 1
    return r


def block_layout(n: int, p: int) -> tuple[int, int]:
    """(rb, r): rows per block and the padded (power-of-two) block size."""
    if p < 1 or p > n:
        raise ValueError("need 1 <= p <= n")
    rb = -(-n // p)
    return rb, next_pow2(rb)


def _sign_bits(seed: int, stream: int, block: int, count: int) -> np.ndarray:
    """+-1 signs for indices 0..count-1 of one (stream, block) pair."""
    calls = (count + 255) // 256
    words = np.array([philox4x64_10((c, block, stream, 0), (seed, 0))
                      for c in range(calls)], dtype=np.uint64).reshape(-1)
    bits = (words[:, None] >> np.arange(64, dtype=np.uint64)[None, :]) & np.uint64(1)
    bits = bits.reshape(-1)[:count]
    return np.where(bits == 1, -1.0, 1.0)


@functools.lru_cache(maxsize=64)
def d_signs(seed: int, block: int, r: int) -> np.ndarray:
    """Diagonal of D^(block), length r."""
    return _sign_bits(seed, STREAM_D, block, r)


@functools.lru_cache(maxsize=64)
def dt_signs(seed: int, block: int, l: int) -> np.ndarray:
    """Diagonal of Dt^(block), length l."""
    return _sign_bits(seed, STREAM_DT, block, l)


@functools.lru_cache(maxsize=16)
def samples(seed: int, l: int, r: int) -> np.ndarray:
    """Row indices s_0..s_{l-1} of the shared sampling matrix R (with replacement)."""
    s = np.empty(l, dtype=np.int64)
    for call in range((l + 3) // 4):
        words = philox4x64_10((call, 0, STREAM_R, 0), (seed, 0))
        for w in range(4):
            j = call * 4 + w
            if j < l:
                s[j] = words[w] % r
    return s


@functools.lru_cache(maxsize=8)
def sylvester(r: int) -> np.ndarray:
    """Unnormalised r x r Hadamard matrix with +-1 entries, Sylvester recursion."""
    if r < 1 or (r & (r - 1)):
        raise ValueError("r must be a power of two")
    h = np.ones((1, 1), dtype=np.int8)
    while h.shape[0] < r:
        h = np.block([[h, h], [h, -h]])
    h.setflags(write=False)
    return h


def _hadamard_rows(rows: np.ndarray, r: int, c0: int, c1: int,
                   inner: int = 4096) -> np.ndarray:
    """Entries H_r[rows, c0:c1] of the unnormalised Hadamard matrix.

    Uses the tensor form of Sec. 2: with r = r1 * r2 (r2 = min(r, inner)),
    H_r = H_{r1} (x) H_{r2}, so H_r[s, a*r2 + b] = H_{r1}[s // r2, a] *
    H_{r2}[s % r2, b]. Both factors come from the Sylvester recursion.
    """
    r2 = min(r, inner)
    r1 = r // r2
    h2 = sylvester(r2)
    h1 = sylvester(r1)
    cols = np.arange(c0, c1)
    outer = h1[np.ix_(rows // r2, cols // r2)].astype(np.float64)
    inner_f = h2[np.ix_(rows % r2, cols % r2)].astype(np.float64)
    return outer * inner_f


def omega_block(n: int, p: int, l: int, seed: int, block: int,
                c0: int = 0, c1: int | None = None) -> np.ndarray:
    """Columns [c0, c1) of Omega^(block) restricted to the block's real rows.

    Returns an l x (c1 - c0) FP64 matrix; column k is local row k of block
    ``block``. Entry (j, k) = sqrt(r/l) * Dt_jj * (H_r[s_j, k] / sqrt(r)) * D_kk.
    """
    rb, r = block_layout(n, p)
    rows_here = max(0, min(n, (block + 1) * rb) - block * rb)
    c1 = rows_here if c1 is None else min(c1, rows_here)
    if c1 <= c0:
        return np.zeros((l, 0))
    s = samples(seed, l, r)
    d = d_signs(seed, block, r)[c0:c1]
    dt = dt_signs(seed, block, l)
    h = _hadamard_rows(s, r, c0, c1)
    scale = math.sqrt(r / l) / math.sqrt(r)
    return scale * (dt[:, None] * h * d[None, :])


def dense_omega(n: int, p: int, l: int, seed: int) -> np.ndarray:
    """The full l x n block SRHT matrix (eq. 2.3), for small n."""
    rb, _ = block_layout(n, p)
    om = np.zeros((l, n))
    for i in range(p):
        r0 = i * rb
        r1 = min(n, r0 + rb)
        if r1 > r0:
            om[:, r0:r1] = omega_block(n, p, l, seed, i)
    return om


def sketch_dense(a: np.ndarray, p: int, l: int, seed: int,
                 chunk: int = 8192) -> np.ndarray:
    """B = Omega A as sum_i Omega^(i) A^(i) (eq. 2.4) with explicit dense blocks.

    ``a`` is n x m; the product is formed in FP64, chunk by chunk of rows,
    so memory stays at l x chunk for Omega.
    """
    a = np.asarray(a)
    n, m = a.shape
    rb, _ = block_layout(n, p)
    out = np.zeros((l, m))
    for i in range(p):
        r0 = i * rb
        r1 = min(n, r0 + rb)
        for k0 in range(0, max(0, r1 - r0), chunk):
            k1 = min(r1 - r0, k0 + chunk)
            om = omega_block(n, p, l, seed, i, k0, k1)
            out += om @ a[r0 + k0:r0 + k1].astype(np.float64)
    return out


def fwht_rows(x: np.ndarray) -> np.ndarray:
    """Unnormalised Walsh-Hadamard transform along axis 0 (natural order).

    Butterflies (u, v) -> (u + v, u - v) over every bit of the row index: one
    2 x 2 Kronecker factor of the tensor form of H (Sec. 2) per bit.
    """
    x = np.array(x, dtype=np.float64, copy=True)
    r = x.shape[0]
    h = 1
    while h < r:
        y = x.reshape(r // (2 * h), 2, h, *x.shape[1:])
        u = y[:, 0].copy()
        v = y[:, 1]
        y[:, 0] += v
        y[:, 1] = u - v
        h *= 2
    return x


def sketch_fast(a: np.ndarray, p: int, l: int, seed: int) -> np.ndarray:
    """Second formulation of Omega A: per block, pad to r rows, flip signs with
    D^(i), apply the FWHT, keep the sampled rows, flip with Dt^(i), sum over
    blocks, scale by 1/sqrt(l). Used to cross-check ``sketch_dense``."""
    a = np.asarray(a)
    n, m = a.shape
    rb, r = block_layout(n, p)
    s = samples(seed, l, r)
    out = np.zeros((l, m))
    for i in range(p):
        r0 = i * rb
        r1 = min(n, r0 + rb)
        x = np.zeros((r, m))
        if r1 > r0:
            x[: r1 - r0] = a[r0:r1]
        x *= d_signs(seed, i, r)[:, None]
        t = fwht_rows(x)
        out += dt_signs(seed, i, l)[:, None] * t[s]
    return out / math.sqrt(l)
