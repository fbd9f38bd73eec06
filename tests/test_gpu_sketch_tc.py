"""Parity of the tensor-core sketch variant (K2, BSRHT_VARIANT_TENSOR) with
the CPU oracle (GPU).

K2 takes 16-bit inputs (BF16, FP16); the +-1 Hadamard operand and the
inputs are exact in the operand type and the products accumulate in FP32, so
the bound is the FP32 one: relative Frobenius error <= 1e-5 against the
FP64 oracle on the same (16-bit) values.  Shapes cover several chunks and
blocks, ragged rows (zero padding) and panels, l above one register group
and above r, row strides, and the full-size 16-bit workload on sampled
columns."""

import numpy as np
import pytest
import torch

from oracle import bsrht as orc
import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_11295_gb300 as b
    return b


def _rel(got, ref):
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(np.asarray(got, dtype=np.float64) - ref) / (den if den > 0 else 1.0)


def _case(lib, n, m, p, l, dtype, seed=0, lda=None):
    a_host = torch.from_numpy(synth.gaussian(n, m, seed=n * 5 + m * 7 + p + l)).to(dtype)
    ref = orc.sketch_fast(a_host.to(torch.float64).numpy(), p, l, seed)
    if lda is not None and lda > m:
        big = torch.zeros(n, lda, dtype=dtype)
        big[:, :m] = a_host
        a_dev = big.cuda()[:, :m]
    else:
        a_dev = a_host.cuda()
    out = lib.bsrht_sketch(a_dev, p, l, seed, variant=lib.VARIANT_TENSOR)
    torch.cuda.synchronize()
    return out.cpu().numpy(), ref


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("n,m,p,l", [
    (4096, 64, 4, 128),     # r = 1024: two chunks per block
    (4096, 100, 1, 300),    # p = 1, ragged panel
    (20000, 33, 3, 200),    # r = 8192, ragged last chunk of each block
    (5000, 17, 7, 96),      # block rows 715 (zero padding inside the chunk)
    (3000, 48, 6, 300),     # r = 512: one partial chunk per block
    (1024, 64, 2, 64),      # r = 512, exact
    (8192, 64, 8, 600),     # l > 512: 64 accumulators per thread
    (8192, 40, 2, 1024),    # l = 1024
    (2048, 8, 2, 1100),     # l > 1024: two sketch-row groups
    (512, 3, 1, 512),       # l = r, sampling with replacement
])
def test_tc_sketch_matches_oracle(lib, dtype, n, m, p, l):
    # TMA needs 16-byte rows: ragged m is stored with its row stride padded to 8.
    lda = None if m % 8 == 0 else (m + 7) // 8 * 8
    got, ref = _case(lib, n, m, p, l, dtype, lda=lda)
    assert got.shape == (l, m)
    assert _rel(got, ref) <= TOL


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_tc_sketch_row_stride(lib, dtype):
    got, ref = _case(lib, 3000, 21, 3, 64, dtype, lda=40)
    assert _rel(got, ref) <= TOL


def test_tc_agrees_with_cuda_core_variant(lib):
    a = torch.from_numpy(synth.gaussian(1 << 16, 160, seed=9)).to(torch.bfloat16).cuda()
    k1 = lib.bsrht_sketch(a, 8, 512, 4, variant=lib.VARIANT_CUDACORE)
    k2 = lib.bsrht_sketch(a, 8, 512, 4, variant=lib.VARIANT_TENSOR)
    torch.cuda.synchronize()
    assert (torch.linalg.norm(k1 - k2) / torch.linalg.norm(k1)).item() <= 1e-5


def test_tc_rejects_what_it_cannot_run(lib):
    """EUNSUP: FP32 input, blocks below one 512-row chunk, rows that break
    the 16-byte TMA stride rule."""
    a32 = torch.zeros(4096, 32, device="cuda", dtype=torch.float32)
    small_r = torch.zeros(2048, 32, device="cuda", dtype=torch.bfloat16)
    odd = torch.zeros(4096, 41, device="cuda", dtype=torch.bfloat16)[:, :40]
    for a, p in ((a32, 4), (small_r, 16), (odd, 4)):
        with pytest.raises(lib.BsrhtError) as e:
            lib.bsrht_sketch(a, p, 64, 0, variant=lib.VARIANT_TENSOR)
        assert e.value.status == -95


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_tc_full_size_sampled_columns(lib, dtype):
    """n = 2^20, m = 8192, p = 8, l = 1024: the 16-bit workload at full size in
    the launch configuration the benchmark times; eight columns are checked
    against the oracle."""
    n, m, p, l = 1 << 20, 8192, 8, 1024
    gen = torch.Generator("cuda").manual_seed(77)
    a = torch.randn(n, m, device="cuda", dtype=torch.float32, generator=gen).to(dtype)
    out = lib.bsrht_sketch(a, p, l, 3, variant=lib.VARIANT_TENSOR)
    cols = [0, 1, 31, 32, 4000, 4095, 8160, 8191]
    sub = a[:, cols].double().cpu().numpy()
    got = out[:, cols].double().cpu().numpy()
    del a
    ref = orc.sketch_fast(sub, p, l, 3)
    assert _rel(got, ref) <= TOL
