"""FP64 arithmetic on FP32 storage (bsrht_opts.precision = BSRHT_PREC_F64).

The sketch of FP32 data is the exact integer Walsh-Hadamard transform of the
FP32 values widened to FP64 (the FP64 kernel), written in FP64: compared
column by column with the CPU oracle applied to the same values in FP64, at
the FP64 bar of 1e-12.  Nystrom (Algorithm 2) of an FP32-stored PSD matrix
then runs in FP64 after the sketch and matches the oracle on the same values
at the FP64 tolerances of test_gpu_lowrank.py; the served request with this
precision gives the direct call's result."""

import numpy as np
import pytest
import torch

from oracle import bsrht as orc
from oracle import lowrank as orl
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_11295_gb300 as b
    return b


def _colwise_rel(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    sc = np.max(np.abs(ref), axis=0)
    sc = np.where(sc > 0, sc, 1.0)
    den = np.linalg.norm(ref / sc, axis=0)
    num = np.linalg.norm((got - ref) / sc, axis=0)
    return np.max(np.where(den > 0, num / np.where(den > 0, den, 1.0), num))


@pytest.mark.parametrize("n,m,p,l", [
    (4096, 256, 4, 128),     # one sketch-row group
    (20000, 36, 3, 300),     # ragged blocks and panels, groups of 512
    (3000, 48, 6, 200),      # chunks straddle the block end (rb = 500)
    (16384, 20, 2, 513),     # two groups
    (2048, 16, 4, 700),      # l > r
])
def test_sketch_f32_storage_f64_arithmetic(lib, n, m, p, l):
    a32 = synth.gaussian(n, m, seed=n + m).astype(np.float32)
    a32[:, 1] *= np.float32(1e-30)  # a column of tiny magnitudes keeps its own scale
    out = lib.bsrht_sketch(torch.from_numpy(a32).cuda(), p, l, 3, precision=lib.PREC_F64)
    torch.cuda.synchronize()
    assert out.dtype == torch.float64 and out.shape == (l, m)
    ref = orc.sketch_fast(a32.astype(np.float64), p, l, 3)
    assert _colwise_rel(out.cpu().numpy(), ref) <= 1e-12


def test_sketch_f32_storage_f64_row_stride(lib):
    a32 = synth.gaussian(6000, 30, seed=8).astype(np.float32)
    big = torch.zeros(6000, 44, dtype=torch.float32)
    big[:, :30] = torch.from_numpy(a32)
    out = lib.bsrht_sketch(big.cuda()[:, :30], 3, 96, 1, precision=lib.PREC_F64)
    torch.cuda.synchronize()
    assert _colwise_rel(out.cpu().numpy(), orc.sketch_fast(a32.astype(np.float64), 3, 96, 1)) <= 1e-12


def test_sketch_f32_storage_f64_is_more_accurate_than_fp32(lib):
    """Against the oracle on the same values: FP64 arithmetic at FP64
    rounding, FP32 arithmetic at FP32 rounding."""
    a32 = synth.lowrank_noise(1 << 15, 64, rank=32, seed=9).astype(np.float32)
    ref = orc.sketch_fast(a32.astype(np.float64), 4, 128, 2)
    a = torch.from_numpy(a32).cuda()
    e64 = _colwise_rel(lib.bsrht_sketch(a, 4, 128, 2, precision=lib.PREC_F64).cpu().numpy(), ref)
    e32 = _colwise_rel(lib.bsrht_sketch(a, 4, 128, 2).double().cpu().numpy(), ref)
    assert e64 <= 1e-12 and e32 > 1e-9


def test_nystrom_f32_storage_f64_matches_oracle(lib):
    """A PSD matrix of rank 400 (eigenvalues 1/i) stored in FP32: with FP64
    arithmetic the rank threshold of Remark 3.1 is the FP64 one, so
    eigenvalues the FP32 path must drop are kept, as in the oracle."""
    n, k, l, p = 1 << 13, 100, 300, 4
    a32 = synth.psd_lowrank(n, 400, seed=31).astype(np.float32)
    a64 = a32.astype(np.float64)
    u, lam = lib.bsrht_nystrom(torch.from_numpy(a32).cuda(), k, l, p, 2, precision=lib.PREC_F64)
    torch.cuda.synchronize()
    u, lam = u.cpu().numpy(), lam.cpu().numpy()
    ur, lr, _ = orl.nystrom(a64, k, l, p, 2)
    assert np.max(np.abs(lam - lr)) <= 1e-10 * lr[0]
    tr = np.trace(a64)
    assert abs(lam.sum() - lr.sum()) <= 1e-10 * tr
    assert np.linalg.norm(u.T @ u - np.eye(k)) <= 1e-10


def test_served_nystrom_f64_precision_equals_direct(lib):
    n, k, l, p = 1 << 13, 60, 200, 4
    a = torch.from_numpy(synth.psd_lowrank(n, 300, seed=32).astype(np.float32)).cuda()
    u0, lam0 = lib.bsrht_nystrom(a, k, l, p, 5, precision=lib.PREC_F64)
    srv = lib.Server(hbm_budget=2 << 30, executors=2)
    try:
        u = torch.empty(n, k, device="cuda", dtype=torch.float64)
        lam = torch.empty(k, device="cuda", dtype=torch.float64)
        t = srv.submit_nystrom(a, k, l, p, 5, (u, lam), precision=lib.PREC_F64)
        assert srv.wait(t) == 0
    finally:
        srv.close()
    torch.cuda.synchronize()
    assert torch.linalg.norm(lam - lam0).item() <= 1e-12 * torch.linalg.norm(lam0).item()


def test_prec_f64_rejected_where_unsupported(lib):
    a = torch.zeros(4096, 64, device="cuda", dtype=torch.float32)
    with pytest.raises(lib.BsrhtError) as e:  # 34 FP32 values per row: rows not on 16 bytes
        lib.bsrht_sketch(torch.zeros(4096, 34, device="cuda", dtype=torch.float32), 4, 64, 0,
                         precision=lib.PREC_F64)
    assert e.value.status == -95
    with pytest.raises(lib.BsrhtError) as e:
        lib.bsrht_sketch(a.to(torch.bfloat16), 4, 64, 0, precision=lib.PREC_F64)
    assert e.value.status == -95
    with pytest.raises(lib.BsrhtError) as e:
        lib.bsrht_sketch(a, 4, 64, 0, variant=lib.VARIANT_TENSOR, precision=lib.PREC_F64)
    assert e.value.status == -95
