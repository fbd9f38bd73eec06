"""Parity of the CUDA block SRHT sketch with the CPU oracle (GPU).

Element-by-element comparison on seeded inputs: relative Frobenius error
<= 1e-12 for FP64 and <= 1e-5 for FP32 arithmetic (bf16/f16 inputs are exact
in FP32, so their bound is the FP32 one).  Sizes span several chunks and
column panels with ragged tails; the full-size cases compare sampled columns
(the sketch is column-separable: (Omega A)[:, J] = Omega A[:, J])."""

import numpy as np
import pytest
import torch

from oracle import bsrht as orc
import synth

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5, torch.bfloat16: 1e-5, torch.float16: 1e-5}


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


def _case(lib, n, m, p, l, dtype, seed=0, lda=None, variant=0):
    a64 = synth.gaussian(n, m, seed=n * 7 + m * 3 + p + l)
    a_host = torch.from_numpy(a64).to(dtype)
    ref = orc.sketch_fast(a_host.to(torch.float64).numpy(), p, l, seed)
    if lda is not None and lda > m:
        big = torch.zeros(n, lda, dtype=dtype)
        big[:, :m] = a_host
        a_dev = big.cuda()[:, :m]
    else:
        a_dev = a_host.cuda()
    out = lib.bsrht_sketch(a_dev, p, l, seed, variant=variant)
    torch.cuda.synchronize()
    return out.cpu().numpy(), ref


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,m,p,l", [
    (4096, 256, 4, 128),      # the small FP64 workload's shape
    (4096, 100, 1, 128),      # p = 1 (standard SRHT times Dt), ragged panel
    (8192, 40, 8, 64),        # r = 1024 = one chunk per block
    (20000, 33, 3, 200),      # r = 8192: several chunks per block, ragged rows
    (5000, 17, 7, 96),        # non-power-of-two block rows (zero padding)
    (3000, 48, 6, 300),       # r = 512
    (2048, 32, 16, 128),      # r = 128
    (1024, 20, 16, 64),       # r = 64 (smallest FP64 chunk)
    (640, 31, 20, 40),        # r = 32 (smallest FP32 chunks / FP64 direct path)
    (256, 9, 64, 32),         # r = 4: direct path for both
    (300, 5, 300, 50),        # r = 1: Rademacher limit
    (2048, 8, 2, 1100),       # l > JG: several sketch-row groups
    (8192, 40, 4, 600),       # 512 < l <= 768: 768-row groups of the 256-thread TMA kernel
    (4096, 24, 2, 768),       # the largest l of those groups
    (4096, 24, 2, 769),       # one more: 1024-row groups
    (512, 3, 4, 512),         # l > r: sampling with replacement
])
def test_sketch_matches_oracle(lib, dtype, n, m, p, l):
    got, ref = _case(lib, n, m, p, l, dtype)
    assert got.shape == (l, m)
    assert _rel(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("n,m,p,l", [(8192, 64, 8, 256), (4096, 50, 2, 128), (1000, 40, 5, 64), (8192, 64, 8, 700)])
def test_sketch_half_inputs(lib, dtype, n, m, p, l):
    got, ref = _case(lib, n, m, p, l, dtype)
    assert _rel(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_sketch_row_stride(lib, dtype):
    got, ref = _case(lib, 3000, 21, 3, 64, dtype, lda=40)
    assert _rel(got, ref) <= TOL[dtype]


def test_sketch_empty_columns(lib):
    a = torch.zeros(64, 0, device="cuda", dtype=torch.float32)
    out = lib.bsrht_sketch(a, 2, 8, 0)
    assert out.shape == (8, 0)


def test_sketch_deterministic(lib):
    a = torch.randn(1 << 15, 96, device="cuda", dtype=torch.float32, generator=torch.Generator("cuda").manual_seed(3))
    b1 = lib.bsrht_sketch(a, 4, 256, 11)
    b2 = lib.bsrht_sketch(a, 4, 256, 11)
    torch.cuda.synchronize()
    assert torch.equal(b1, b2)


def test_sketch_block_additivity(lib):
    """eq. 2.4 on the device: one launch over p blocks equals the sum of p
    launches that each see one block (the others zeroed)."""
    n, m, p, l = 1 << 14, 64, 4, 128
    a = torch.randn(n, m, device="cuda", dtype=torch.float64, generator=torch.Generator("cuda").manual_seed(5))
    full = lib.bsrht_sketch(a, p, l, 2)
    rb = n // p
    acc = torch.zeros_like(full)
    for i in range(p):
        ai = torch.zeros_like(a)
        ai[i * rb:(i + 1) * rb] = a[i * rb:(i + 1) * rb]
        acc += lib.bsrht_sketch(ai, p, l, 2)
    torch.cuda.synchronize()
    assert (torch.linalg.norm(acc - full) / torch.linalg.norm(full)).item() <= 1e-13


@pytest.mark.parametrize("p", [1, 4, 16, 64])
def test_sketch_full_size_sampled_columns(lib, p):
    """n = 2^20, m = 4096, l = 512 in FP32, the tall-skinny workload at full
    size in the launch configuration the benchmark times; eight columns
    (first, last and spread) are checked against the oracle."""
    n, m, l = 1 << 20, 4096, 512
    gen = torch.Generator("cuda").manual_seed(100 + p)
    a = torch.randn(n, m, device="cuda", dtype=torch.float32, generator=gen)
    out = lib.bsrht_sketch(a, p, l, 7)
    cols = [0, 1, 31, 32, 1000, 2047, 4064, 4095]
    sub = a[:, cols].double().cpu().numpy()
    got = out[:, cols].double().cpu().numpy()
    del a
    ref = orc.sketch_fast(sub, p, l, 7)
    assert _rel(got, ref) <= 1e-5


@pytest.mark.parametrize("p", [4, 64])
def test_sketch_full_size_sampled_columns_fp64(lib, p):
    """n = 2^20, m = 4096, l = 512 in FP64 (the paper's arithmetic), the
    launch configuration of the FP64 benchmark line; eight columns (first,
    last, panel edges, spread) against the oracle at 1e-12."""
    n, m, l = 1 << 20, 4096, 512
    gen = torch.Generator("cuda").manual_seed(200 + p)
    a = torch.randn(n, m, device="cuda", dtype=torch.float64, generator=gen)
    out = lib.bsrht_sketch(a, p, l, 9)
    cols = [0, 1, 15, 16, 1000, 2047, 4080, 4095]
    sub = a[:, cols].cpu().numpy()
    got = out[:, cols].cpu().numpy()
    del a
    ref = orc.sketch_fast(sub, p, l, 9)
    assert _rel(got, ref) <= 1e-12
