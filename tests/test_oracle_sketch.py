"""Pins of the CPU oracle's sketch against what the paper and the mathematics
fix (no GPU). Each test names the passage it checks."""

import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import bsrht
from oracle.philox import philox4x64_10
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox
@pytest.mark.parametrize("counter,key", [
    ((1, 0, 0, 0), (0, 0)),
    ((7, 3, 2, 0), (12345, 0)),
    ((0, 5, 1, 0), (2**64 - 1, 0)),
    ((2**64 - 1, 9, 0, 0), (42, 7)),       # carry into the second word
])
def test_philox_matches_numpy(counter, key):
    """Our Philox4x64-10 against numpy's independent implementation.
    numpy advances the 256-bit counter before each block."""
    c = sum(int(w) << (64 * i) for i, w in enumerate(counter)) - 1
    start = np.array([(c >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=start)
    ref = [int(x) for x in bg.random_raw(4)]
    assert list(philox4x64_10(counter, key)) == ref


# ---------------------------------------------------------------- Hadamard
@pytest.mark.parametrize("r", [1, 2, 4, 8, 64, 256, 1024])
def test_sylvester_orthogonal(r):
    """H H^T = r I for the unnormalised matrix (so H / sqrt(r) is orthogonal)."""
    h = bsrht.sylvester(r).astype(np.int64)
    assert np.array_equal(h @ h.T, r * np.eye(r, dtype=np.int64))


@pytest.mark.parametrize("r", [2, 16, 128, 512])
def test_sylvester_closed_form_and_scipy(r):
    """Entries are (-1)^popcount(a & b); scipy.linalg.hadamard builds the same matrix."""
    h = bsrht.sylvester(r)
    a = np.arange(r)
    pc = np.array([[bin(x & y).count("1") & 1 for y in a] for x in a])
    assert np.array_equal(h, np.where(pc == 1, -1, 1))
    assert np.array_equal(h, sla.hadamard(r))


def test_tensor_form_from_paper_factor():
    """Sec. 2: H_r = H2 (x) ... (x) H2 with the printed 2 x 2 factor."""
    h2 = np.loadtxt(os.path.join(GOLDEN, "hadamard_factor.txt"), dtype=np.int64)
    h = np.ones((1, 1), dtype=np.int64)
    for r in (2, 4, 8, 16, 32):
        h = np.kron(h2, h)
        assert np.array_equal(h, bsrht.sylvester(r))


def test_hadamard_rows_large_r():
    """Kronecker-split rows of H_r for r > inner size agree with the closed form."""
    r = 1 << 14
    rng = np.random.default_rng(0)
    rows = rng.integers(0, r, size=12)
    c0, c1 = 5000, 5300
    got = bsrht._hadamard_rows(rows, r, c0, c1, inner=256)
    cols = np.arange(c0, c1)
    pc = np.array([[bin(int(s) & int(k)).count("1") & 1 for k in cols] for s in rows])
    assert np.array_equal(got, np.where(pc == 1, -1.0, 1.0))


# ---------------------------------------------------------------- Omega
def _brute_omega(n, p, l, seed):
    """eq. 2.3 assembled from explicit matrices: sqrt(r/l) Dt R H D per block,
    with H = scipy.linalg.hadamard(r) / sqrt(r) and R an l x r selection."""
    rb, r = bsrht.block_layout(n, p)
    s = bsrht.samples(seed, l, r)
    rmat = np.zeros((l, r))
    rmat[np.arange(l), s] = 1.0
    h = sla.hadamard(r) / math.sqrt(r)
    blocks = []
    for i in range(p):
        rows = max(0, min(n, (i + 1) * rb) - i * rb)
        full = math.sqrt(r / l) * (np.diag(bsrht.dt_signs(seed, i, l)) @ rmat @ h
                                   @ np.diag(bsrht.d_signs(seed, i, r)))
        blocks.append(full[:, :rows])
    return np.hstack(blocks)


@pytest.mark.parametrize("n,p,l,seed", [
    (16, 4, 8, 0), (16, 1, 8, 3), (13, 3, 5, 1), (16, 16, 6, 2), (9, 4, 12, 7), (10, 2, 3, 11),
])
def test_brute_force_omega(n, p, l, seed):
    om = bsrht.dense_omega(n, p, l, seed)
    assert om.shape == (l, n)
    np.testing.assert_allclose(om, _brute_omega(n, p, l, seed), rtol=0, atol=1e-15)
    assert np.allclose(np.abs(om), 1.0 / math.sqrt(l))


def test_golden_regression_omega():
    """Fixture written by tests/golden/make_golden.py (oracle only): freezes the
    Philox layout of the signs and samples."""
    data = np.loadtxt(os.path.join(GOLDEN, "omega_n16_p4_l8_seed0.txt"), dtype=np.int64)
    om = bsrht.dense_omega(16, 4, 8, 0)
    assert np.array_equal(np.sign(om).astype(np.int64), data)


def test_p1_reduces_to_srht():
    """Sec. 2: with p = 1 the block SRHT is Dt times the standard SRHT of
    eq. 2.1, sqrt(n/l) R H D, built independently here."""
    n, l, seed = 64, 24, 5
    om = bsrht.dense_omega(n, 1, l, seed)
    s = bsrht.samples(seed, l, n)
    d = bsrht.d_signs(seed, 0, n)
    srht = math.sqrt(n / l) * (sla.hadamard(n) / math.sqrt(n))[s] * d[None, :]
    dt = bsrht.dt_signs(seed, 0, l)
    np.testing.assert_allclose(om, dt[:, None] * srht, atol=1e-15)
    np.testing.assert_allclose(om.T @ om, srht.T @ srht, atol=1e-13)


def test_r1_reduces_to_rademacher():
    """Sec. 2: with r = 1 (p = n) the block SRHT is a Rademacher matrix: every
    entry +-1/sqrt(l), independent across rows and columns (full rank)."""
    n, l = 48, 20
    om = bsrht.dense_omega(n, n, l, 3)
    assert np.allclose(np.abs(om), 1 / math.sqrt(l))
    assert np.linalg.matrix_rank(om) == min(n, l)
    assert abs(om.mean()) < 5.0 / math.sqrt(l) / math.sqrt(n * l)
    assert len({tuple(np.sign(row)) for row in om}) == l


@pytest.mark.parametrize("n,m,p,l", [
    (256, 7, 4, 32), (300, 5, 3, 40), (1000, 3, 8, 200), (64, 4, 64, 16),
    (128, 6, 1, 300), (17, 2, 5, 17), (4096, 2, 2, 128),
])
def test_dense_and_fast_sketch_agree(n, m, p, l):
    """Two formulations of eq. 2.4: explicit dense blocks vs FWHT + sampling."""
    a = synth.gaussian(n, m, seed=n + m + p + l)
    b1 = bsrht.sketch_dense(a, p, l, seed=9)
    b2 = bsrht.sketch_fast(a, p, l, seed=9)
    assert np.linalg.norm(b1 - b2) <= 1e-13 * np.linalg.norm(b1)


def test_block_additivity():
    """eq. 2.4: Omega A is the sum of the per-block contributions."""
    n, m, p, l = 512, 3, 4, 64
    a = synth.gaussian(n, m, seed=1)
    rb, _ = bsrht.block_layout(n, p)
    total = np.zeros((l, m))
    for i in range(p):
        ai = np.zeros_like(a)
        ai[i * rb:(i + 1) * rb] = a[i * rb:(i + 1) * rb]
        total += bsrht.sketch_fast(ai, p, l, seed=4)
    np.testing.assert_allclose(total, bsrht.sketch_fast(a, p, l, seed=4), atol=1e-12)


def test_isometry_in_expectation():
    """E[Omega^T Omega] = I: the diagonal is exactly 1 (entries +-1/sqrt(l)) and
    the off-diagonal entries average to 0 over seeds (Monte Carlo)."""
    n, p, l, trials = 32, 4, 8, 600
    acc = np.zeros((n, n))
    acc2 = np.zeros((n, n))
    for seed in range(trials):
        om = bsrht.dense_omega(n, p, l, seed)
        g = om.T @ om
        np.testing.assert_allclose(np.diag(g), 1.0, atol=1e-14)
        acc += g
        acc2 += g * g
    mean = acc / trials
    sd = np.sqrt(np.maximum(acc2 / trials - mean ** 2, 1e-30))
    off = ~np.eye(n, dtype=bool)
    z = np.abs(mean[off]) / (sd[off] / math.sqrt(trials))
    assert np.max(z) < 5.0


@pytest.mark.parametrize("p", [1, 4, 16])
def test_subspace_embedding_distortion(p):
    """Def. 1.1 / Thm 2.1 (empirically): singular values of Omega V for an
    orthonormal V stay in the Marchenko-Pastur-like band 1 +- 1.5 sqrt(d/l),
    as a Gaussian embedding of the same size does."""
    n, d, l = 2048, 10, 128
    rng = np.random.default_rng(10 + p)
    v = synth.haar(n, d, rng)
    band = 1.5 * math.sqrt(d / l)
    worst = 0.0
    for seed in range(4):
        sv = np.linalg.svd(bsrht.sketch_fast(v, p, l, seed), compute_uv=False)
        worst = max(worst, np.max(np.abs(sv - 1.0)))
    assert worst < band


def test_sampling_with_replacement_and_range():
    """Sec. 2: R samples with replacement from [0, r); l > r is allowed."""
    s = bsrht.samples(1, 500, 64)
    assert s.min() >= 0 and s.max() < 64
    assert len(np.unique(s)) < 500
    counts = np.bincount(s, minlength=64)
    # chi-square goodness of fit for uniform sampling (df = 63; 99.9% point ~ 104)
    exp = 500 / 64
    assert np.sum((counts - exp) ** 2 / exp) < 104
