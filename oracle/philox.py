"""Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC'11), written from the published round function.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

One call maps a 256-bit counter (four 64-bit words) and a 128-bit key (two
64-bit words) to four 64-bit outputs through ten rounds. A round multiplies
counter words 0 and 2 by two fixed odd constants, keeps the 128-bit products
as (hi, lo) pairs and permutes/xors them with the other counter words and the
key; between rounds the key is bumped by two Weyl constants.

Pinned in the tests against ``numpy.random.Philox``, an independent
implementation of the same generator (numpy advances its counter by one
before each block, so block c of ours is numpy's stream started at c - 1).
"""

MASK64 = (1 << 64) - 1
# Round multipliers and key-schedule (Weyl) constants of Philox4x64.
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B


def philox4x64_10(counter, key):
    """Return the four 64-bit outputs for ``counter`` (4 words) and ``key`` (2 words)."""
    c0, c1, c2, c3 = (int(w) & MASK64 for w in counter)
    k0, k1 = (int(w) & MASK64 for w in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + PHILOX_W0) & MASK64
            k1 = (k1 + PHILOX_W1) & MASK64
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> 64) ^ c1 ^ k0, p1 & MASK64,
                          (p0 >> 64) ^ c3 ^ k1, p0 & MASK64)
    return (c0, c1, c2, c3)
