"""Oracle parity of Algorithm 1 at the kernel instances the benchmark
configurations run (GPU).

* Tall-skinny FP32 case: n = 2^17 rows of the n = 2^20, m = 4096 workload
  generator (G1 diag(i^-2) G2^T + 1e-4 N), p = 4, l = 512, k = 100 -- the
  TMA-fed sketch with 512-row groups, the 128 x 256 tcgen05 tiles of A Q at
  K = 4096, the l = 512 block Jacobi and the FP32 CholeskyQR2 chain, as at
  full size.
* 16-bit case (BF16 and FP16 storage, FP32 arithmetic): m = 8192 columns,
  p = 8, l = 1024, k = 200 on n = 2^15 rows -- 1024-row sketch groups, the
  scalar FP32 Jacobi (l > 512) and the l = 1024 FP64 polish.

Tolerances (FP32 arithmetic, per the spec bar of 1e-5 on the sketch):
sketch relative Frobenius <= 1e-5 against the oracle on the same stored
values; singular values within 2e-5 sigma_1; the residual ||A - U S V^T||_F
within 1e-4 of the oracle's (relative); orthonormal factors to 1e-4 (U) and
1e-10 (V, built from the FP64 basis of the sketch).  The rank-k factors
themselves are not compared: at these noise levels sigma_k and sigma_{k+1}
are within rounding of each other."""

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


def _resid(a64, u, s, v):
    return float(np.linalg.norm(a64 - (u * s) @ v.T))


def _compare(lib, a_dev, k, l, p, seed):
    a64 = a_dev.double().cpu().numpy()
    b = lib.bsrht_sketch(a_dev, p, l, seed)
    u, s, v = lib.bsrht_rsvd(a_dev, k, l, p, seed)
    torch.cuda.synchronize()
    b = b.double().cpu().numpy()
    u, s, v = u.cpu().numpy(), s.cpu().numpy(), v.cpu().numpy()
    b_ref = orc.sketch_fast(a64, p, l, seed)
    ur, sr, vr = orl.rsvd(a64, k, l, p, seed)
    sk_err = np.linalg.norm(b - b_ref) / np.linalg.norm(b_ref)
    e, e_ref = _resid(a64, u, s, v), _resid(a64, ur, sr, vr)
    return a64, sk_err, (u, s, v), (ur, sr, vr), e, e_ref


def test_rsvd_tall_skinny_fp32_matches_oracle(lib):
    n, m, p, l, k = 1 << 17, 4096, 4, 512, 100
    a = synth.lowrank_noise_device(n, m, seed=1236, dtype=torch.float32)
    _, sk_err, (u, s, v), (ur, sr, vr), e, e_ref = _compare(lib, a, k, l, p, 0)
    assert sk_err <= 1e-5
    assert np.max(np.abs(s - sr)) <= 2e-5 * sr[0]
    assert abs(e - e_ref) <= 1e-4 * e_ref
    assert np.linalg.norm(u.T @ u - np.eye(k)) <= 1e-4
    assert np.linalg.norm(v.T @ v - np.eye(k)) <= 1e-10


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_rsvd_16bit_l1024_matches_oracle(lib, dtype):
    n, m, p, l, k = 1 << 15, 8192, 8, 1024, 200
    a32 = synth.lowrank_noise_device(n, m, seed=1237, dtype=torch.float32)
    a = a32.to(dtype)
    del a32
    _, sk_err, (u, s, v), (ur, sr, vr), e, e_ref = _compare(lib, a, k, l, p, 1)
    assert sk_err <= 1e-5
    assert np.max(np.abs(s - sr)) <= 2e-5 * sr[0]
    assert abs(e - e_ref) <= 1e-4 * e_ref
    assert np.linalg.norm(u.T @ u - np.eye(k)) <= 1e-4
    assert np.linalg.norm(v.T @ v - np.eye(k)) <= 1e-10
