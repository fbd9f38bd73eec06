"""Single-view RSVD (Algorithm 3, bsrht_srsvd) on the GPU against the CPU
oracle (oracle.lowrank.srsvd), through the C ABI.

What is unique is compared: for A of exact (or near-exact) rank below l the
bases Q, P capture range(A) on both sides and the outputs are determined, so
the FP64 path matches the oracle to rounding (1e-12, on exact recovery and
against the oracle on a near-low-rank matrix); for
FP32 data the reduced-precision bar applies (singular values within
2e-5 sigma_1, residuals within 1e-5 ||A||_F, orthonormal factors to 1e-5).  At the full benchmark size: orthonormal factors, descending S and an
error within 1.5x of Algorithm 1's on the same data."""

import numpy as np
import pytest
import torch

from oracle import lowrank as orl
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_11295_gb300 as b
    return b


@pytest.mark.parametrize("p", [1, 4])
def test_srsvd_exact_recovery_fp64(lib, p):
    a = synth.exact_rank(3000, 512, 12, seed=20 + p)
    k, l, s = 12, 30, 64
    u, sv, v = lib.bsrht_srsvd(torch.from_numpy(a).cuda(), k, l, s, p, 5)
    torch.cuda.synchronize()
    u, sv, v = u.cpu().numpy(), sv.cpu().numpy(), v.cpu().numpy()
    assert np.linalg.norm(a - (u * sv) @ v.T) <= 1e-12 * np.linalg.norm(a)
    assert np.linalg.norm(u.T @ u - np.eye(k)) <= 1e-12
    assert np.linalg.norm(v.T @ v - np.eye(k)) <= 1e-12
    ref = np.linalg.svd(a, compute_uv=False)[:k]
    np.testing.assert_allclose(sv, ref, rtol=1e-10, atol=1e-12 * ref[0])


def test_srsvd_matches_oracle_fp64(lib):
    """Rank 10 plus a 1e-9 noise floor: Q and P are rank-revealing bases on
    both sides (every direction above l 2^-44 sigma_1 kept), so both
    determine the same rank-10 factors: 1e-12 relative."""
    rng = np.random.default_rng(30)
    a = synth.exact_rank(4096, 1024, 10, seed=31) + 1e-9 * rng.standard_normal((4096, 1024))
    k, l, s, p = 10, 40, 96, 4
    u, sv, v = lib.bsrht_srsvd(torch.from_numpy(a).cuda(), k, l, s, p, 3)
    torch.cuda.synchronize()
    u, sv, v = u.cpu().numpy(), sv.cpu().numpy(), v.cpu().numpy()
    ur, sr, vr = orl.srsvd(a, k, l, s, p, 3)
    assert np.max(np.abs(sv - sr)) <= 1e-12 * sr[0]
    approx, ref = (u * sv) @ v.T, (ur * sr) @ vr.T
    assert np.linalg.norm(approx - ref) <= 1e-12 * np.linalg.norm(ref)


def test_srsvd_fp32_matches_oracle(lib):
    """FP32 data: a rank-20 signal (sigma_i = i^-2) over a 1e-7 noise floor.
    With l samples drawn with replacement some rows of Gamma repeat, X loses
    rank and both sides complete P with arbitrary directions; those carry
    only the noise here, so the outputs agree to the FP32 bar."""
    a32 = synth.lowrank_noise(1 << 15, 384, rank=20, noise=1e-7, seed=12, dtype=np.float32)
    a64 = a32.astype(np.float64)
    k, l, s, p = 20, 64, 128, 4
    u, sv, v = lib.bsrht_srsvd(torch.from_numpy(a32).cuda(), k, l, s, p, 3)
    torch.cuda.synchronize()
    u, sv, v = u.cpu().numpy(), sv.cpu().numpy(), v.cpu().numpy()
    ur, sr, vr = orl.srsvd(a64, k, l, s, p, 3)
    assert np.max(np.abs(sv - sr)) <= 2e-5 * sr[0]
    err = np.linalg.norm(a64 - (u * sv) @ v.T)
    err_ref = np.linalg.norm(a64 - (ur * sr) @ vr.T)
    assert abs(err - err_ref) <= 1e-5 * np.linalg.norm(a64)
    assert np.linalg.norm(u.T @ u - np.eye(k)) <= 1e-5
    assert np.linalg.norm(v.T @ v - np.eye(k)) <= 1e-5


def test_srsvd_full_size_properties(lib):
    """n = 2^20, m = 4096, FP32, k = 100, l = 512, s = 1024, p = 4 (the
    benchmark's workload): orthonormal factors, descending S, sigma_1 of the
    signal, and ||A - U S V^T||_F within 1.5x of Algorithm 1's, the residual
    formed as ||A||^2 - 2 tr(S U^T A V) + ||S||^2 (orthonormal U, V)."""
    n, m, k, l, s, p = 1 << 20, 4096, 100, 512, 1024, 4
    a = synth.lowrank_noise_device(n, m, seed=1236, dtype=torch.float32)

    def resid(u, sv, v):
        av = torch.cat([(a[i:i + 65536].double() @ v) for i in range(0, n, 65536)])
        a2 = sum(float((a[i:i + 65536].double() ** 2).sum()) for i in range(0, n, 65536))
        cross = float(((u.T @ av).diagonal() * sv).sum())
        return max(a2 - 2 * cross + float((sv ** 2).sum()), 0.0) ** 0.5

    u, sv, v = lib.bsrht_srsvd(a, k, l, s, p, 0)
    torch.cuda.synchronize()
    eye = torch.eye(k, device="cuda", dtype=torch.float64)
    assert torch.linalg.norm(u.T @ u - eye).item() <= 1e-4
    assert torch.linalg.norm(v.T @ v - eye).item() <= 1e-10
    sc = sv.cpu().numpy()
    assert np.all(np.diff(sc) <= 0) and sc[-1] >= 0
    assert 0.9 < sc[0] < 1.3
    e_single = resid(u, sv, v)
    ur, sr, vr = lib.bsrht_rsvd(a, k, l, p, 0)
    torch.cuda.synchronize()
    e_two = resid(ur, sr, vr)
    assert e_two <= e_single <= 1.5 * e_two


def test_srsvd_rejects(lib):
    a16 = torch.zeros(512, 64, device="cuda", dtype=torch.bfloat16)
    with pytest.raises(lib.BsrhtError) as e:
        lib.bsrht_srsvd(a16, 4, 8, 16, 1, 0)
    assert e.value.status == -95
    a = torch.zeros(512, 64, device="cuda", dtype=torch.float32)
    for k, l, s in ((4, 8, 65), (4, 16, 8), (9, 8, 16)):  # s > m, l > s, k > l
        with pytest.raises(lib.BsrhtError) as e:
            lib.bsrht_srsvd(a, k, l, s, 1, 0)
        assert e.value.status == -22
