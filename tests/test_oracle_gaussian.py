"""Pins of the Gaussian-embedding oracle (the comparator of Sec. 4) against
what fixes it from outside: the scalar Philox4x64-10 (itself pinned against
numpy's Philox in test_oracle_sketch), the uniform and normal laws
(Kolmogorov-Smirnov), E[Omega^T Omega] = I and the Marchenko-Pastur edges of
a Gaussian embedding of a d-dimensional subspace."""

import numpy as np
import pytest
from scipy import stats

from oracle import gaussian as g
from oracle.philox import philox4x64_10


def test_vectorised_philox_equals_scalar():
    rng = np.random.default_rng(3)
    cs = rng.integers(0, 2**63, size=(64, 4), dtype=np.uint64)
    cs[:5] = [[0, 0, 0, 0], [2**64 - 1, 2**64 - 1, 2**64 - 1, 2**64 - 1], [1, 0, 3, 0], [0, 7, 3, 0], [5, 5, 5, 5]]
    for seed in (0, 1, 12345, 2**64 - 1):
        v = g.philox4x64_10_vec(cs[:, 0], cs[:, 1], cs[:, 2], cs[:, 3], seed, 0)
        for i in range(len(cs)):
            assert tuple(int(v[t][i]) for t in range(4)) == philox4x64_10(tuple(int(x) for x in cs[i]), (seed, 0))


@pytest.mark.parametrize("n,l,seed", [(1, 1, 0), (37, 5, 7), (64, 3, 99)])
def test_entries_follow_the_counter_rule(n, l, seed):
    """Every entry from the vectorised path equals the one-entry scalar path:
    counter (k >> 1, j, 3, 0), words (0, 1) for even k and (2, 3) for odd k."""
    om = g.omega_gaussian(n, l, seed)
    assert om.shape == (l, n)
    for j in range(l):
        for k in range(n):
            assert om[j, k] == pytest.approx(g.omega_gaussian_entry(j, k, l, seed), rel=0, abs=1e-15)


def test_uniforms_are_exact_and_uniform():
    rng = np.random.default_rng(4)
    w = rng.integers(0, 2**64 - 1, size=200000, dtype=np.uint64, endpoint=True)
    u = g.uniform_from_word(w)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.all(u.astype(np.float32).astype(np.float64) == u)  # same value in FP32 and FP64
    assert g.uniform_from_word(np.array([0], dtype=np.uint64))[0] == 2.0**-24
    assert g.uniform_from_word(np.array([2**64 - 1], dtype=np.uint64))[0] == 1.0 - 2.0**-24
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_entries_are_standard_normal_scaled():
    l = 50
    om = g.omega_gaussian(4000, l, 11) * np.sqrt(l)  # 200000 draws of N(0, 1)
    z = om.ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-3
    nz = z.size
    assert abs(z.mean()) < 5 / np.sqrt(nz)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / nz)
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 5 * np.sqrt(24.0 / nz)
    # Even and odd columns use different words of the same Philox block; rows
    # different counters: no correlation between neighbours.
    for a, b in ((om[:, 0::2][:, :1999].ravel(), om[:, 1::2][:, :1999].ravel()), (om[:-1].ravel(), om[1:].ravel())):
        assert abs(np.corrcoef(a, b)[0, 1]) < 5 / np.sqrt(a.size)


def test_seed_determines_omega():
    a = g.omega_gaussian(100, 8, 5)
    assert np.array_equal(a, g.omega_gaussian(100, 8, 5))
    assert not np.allclose(a, g.omega_gaussian(100, 8, 6))


def test_expected_gram_is_identity():
    """E[Omega^T Omega] = I: diagonal and off-diagonal within 4 standard
    errors over 600 seeds (n = 12, l = 4)."""
    n, l, reps = 12, 4, 600
    acc = np.zeros((n, n))
    acc2 = np.zeros((n, n))
    for s in range(reps):
        om = g.omega_gaussian(n, l, 1000 + s)
        gm = om.T @ om
        acc += gm
        acc2 += gm * gm
    mean = acc / reps
    se = np.sqrt(np.maximum(acc2 / reps - mean**2, 1e-30) / reps)
    assert np.all(np.abs(mean - np.eye(n)) < 4 * se + 1e-12)


def test_embedding_within_marchenko_pastur_edges():
    """Singular values of Omega V for an orthonormal V (n x d) fill
    [1 - sqrt(d/l), 1 + sqrt(d/l)] up to O(l^-2/3) fluctuations."""
    n, d, l = 4096, 10, 256
    v, _ = np.linalg.qr(np.random.default_rng(7).standard_normal((n, d)))
    lo, hi = 1 - np.sqrt(d / l), 1 + np.sqrt(d / l)
    for seed in range(3):
        sv = np.linalg.svd(g.omega_gaussian(n, l, seed) @ v, compute_uv=False)
        assert sv.max() < hi + 0.08 and sv.min() > lo - 0.08
        assert sv.max() > 1.0 and sv.min() < 1.0


def test_sketch_is_omega_times_a_in_any_panel_split():
    rng = np.random.default_rng(8)
    a = rng.standard_normal((1000, 7))
    ref = g.omega_gaussian(1000, 16, 3) @ a
    for panel in (1, 64, 999, 1 << 14):
        assert np.allclose(g.gaussian_sketch(a, 16, 3, row_panel=panel), ref, rtol=0, atol=1e-12)
