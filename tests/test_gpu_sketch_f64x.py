"""Parity of the FP64 sketch kernel with the exact integer transform
(16-column panels, 512-row chunks, TMA-fed; taken for FP64 A whose rows are
16-byte aligned and whose blocks hold at least 512 rows) with the CPU oracle.

The transform itself is exact (64-bit integers); the only rounding is the
conversion of each value to fixed point with 48 fraction bits below its
column's scale (and the FP64 adds of the flushed sums), so every column of
the sketch is compared on its own, relative to that column's norm, at 1e-12.
Cases: ragged panels and blocks, one to several sketch-row groups,
magnitudes spread over hundreds of binades between columns and within a
column (the scale grows mid-panel), subnormals, zeros, Inf / NaN columns."""

import numpy as np
import pytest
import torch

from oracle import bsrht as orc
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_11295_gb300 as b
    return b


def _colwise_rel(got, ref):
    """Largest relative Frobenius error over the columns (each column scaled
    by its largest |entry| first, so norms of 1e300-sized columns do not
    overflow)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    sc = np.max(np.abs(ref), axis=0)
    sc = np.where(sc > 0, sc, 1.0)
    den = np.linalg.norm(ref / sc, axis=0)
    num = np.linalg.norm((got - ref) / sc, axis=0)
    return np.max(np.where(den > 0, num / np.where(den > 0, den, 1.0), num))


def _run(lib, a64, p, l, seed, lda=None):
    n, m = a64.shape
    if lda is not None and lda > m:
        big = torch.zeros(n, lda, dtype=torch.float64)
        big[:, :m] = torch.from_numpy(a64)
        a_dev = big.cuda()[:, :m]
    else:
        a_dev = torch.from_numpy(a64).cuda()
    out = lib.bsrht_sketch(a_dev, p, l, seed)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("n,m,p,l", [
    (4096, 256, 4, 128),       # the small FP64 workload (r = 1024, groups of 256)
    (8192, 40, 8, 64),         # one chunk per block, ragged panel (40 = 2 x 16 + 8)
    (20000, 34, 3, 300),       # several chunks per block, ragged block rows, groups of 512
    (3000, 48, 6, 200),        # rb = 500 < 512: chunks straddle the block end
    (65536, 64, 16, 512),      # a full 512-row group
    (16384, 18, 2, 513),       # two groups, the second of one row
    (4096, 32, 2, 1100),       # three groups
    (1 << 15, 2, 1, 1),        # l = 1, p = 1 (the SRHT of eq. 2.1 times Dt)
    (2048, 16, 4, 700),        # l > r: sampling with replacement
])
def test_f64x_matches_oracle(lib, n, m, p, l):
    a = synth.gaussian(n, m, seed=n + m + p + l)
    got = _run(lib, a, p, l, seed=3)
    ref = orc.sketch_fast(a, p, l, 3)
    assert got.shape == (l, m)
    assert _colwise_rel(got, ref) <= 1e-12


def test_f64x_row_stride(lib):
    a = synth.gaussian(6000, 30, seed=8)
    got = _run(lib, a, 3, 96, seed=1, lda=42)
    assert _colwise_rel(got, orc.sketch_fast(a, 3, 96, 1)) <= 1e-12


def test_f64x_column_scales_far_apart(lib):
    """Columns scaled by 1e-300 ... 1e300 (and one subnormal column): each
    keeps its own fixed-point scale."""
    n, m, p, l = 8192, 32, 4, 128
    a = synth.gaussian(n, m, seed=11)
    scales = 10.0 ** np.linspace(-300, 300, m)
    a = a * scales
    a[:, 5] = synth.gaussian(n, 1, seed=12)[:, 0] * 1e-310  # subnormal column
    got = _run(lib, a, p, l, seed=2)
    ref = orc.sketch_fast(a, p, l, 2)
    assert _colwise_rel(np.delete(got, 5, 1), np.delete(ref, 5, 1)) <= 1e-12
    # Subnormal inputs have fewer significant bits themselves; the column is
    # still right to its own precision.
    assert _colwise_rel(got[:, 5:6], ref[:, 5:6]) <= 1e-9


def test_f64x_scale_grows_within_a_panel(lib):
    """Row magnitudes rising by 1e8 per 4096 rows (and a zero stretch): the
    column scale grows chunk after chunk, each time after the integer sums
    at the old scale were flushed."""
    n, m, p, l = 1 << 16, 16, 2, 256
    a = synth.gaussian(n, m, seed=13)
    a *= (10.0 ** (8 * (np.arange(n) // 4096) / 16.0))[:, None]
    a[1000:3000] = 0.0
    got = _run(lib, a, p, l, seed=4)
    ref = orc.sketch_fast(a, p, l, 4)
    assert _colwise_rel(got, ref) <= 1e-12


def test_f64x_heavy_tails(lib):
    """Student-t (3 dof) entries: a few values far above the rest."""
    rng = np.random.default_rng(14)
    a = rng.standard_t(3, size=(1 << 15, 48))
    got = _run(lib, a, 8, 256, seed=5)
    assert _colwise_rel(got, orc.sketch_fast(a, 8, 256, 5)) <= 1e-12


def test_f64x_nonfinite_columns(lib):
    """An Inf in column 3 and a NaN in column 20 make exactly those sketch
    columns NaN; the other columns are unaffected."""
    n, m, p, l = 4096, 32, 4, 64
    a = synth.gaussian(n, m, seed=15)
    a[777, 3] = np.inf
    a[4000, 20] = np.nan
    got = _run(lib, a, p, l, seed=6)
    assert np.all(np.isnan(got[:, 3])) and np.all(np.isnan(got[:, 20]))
    keep = [c for c in range(m) if c not in (3, 20)]
    b = a.copy()
    b[:, 3] = 0.0
    b[:, 20] = 0.0
    ref = orc.sketch_fast(b, p, l, 6)
    assert np.all(np.isfinite(got[:, keep]))
    assert _colwise_rel(got[:, keep], ref[:, keep]) <= 1e-12


def test_f64x_zero_matrix(lib):
    got = _run(lib, np.zeros((4096, 16)), 2, 32, seed=1)
    assert np.all(got == 0.0)


def test_f64x_deterministic(lib):
    a = torch.randn(1 << 16, 48, device="cuda", dtype=torch.float64, generator=torch.Generator("cuda").manual_seed(9))
    b1 = lib.bsrht_sketch(a, 4, 384, 12)
    b2 = lib.bsrht_sketch(a, 4, 384, 12)
    torch.cuda.synchronize()
    assert torch.equal(b1, b2)
