"""Parity of the CUDA randomized SVD (Algorithm 1) and Nystrom (Algorithm 2)
with the CPU oracle on the same seeded inputs (GPU).

Tolerances. FP64 inputs: the rank-k approximation U S V^T and the singular
values to 1e-12 relative (the rank-revealing basis of range(Y) makes the
result unique; CholeskyQR2 and Jacobi vs Householder and LAPACK SVD differ
only by rounding); Nystrom eigenvalues to 1e-10 relative to the largest. FP32 inputs: the tall products run in
FP32, so values agree to 2e-5 relative to the largest and approximation
errors to 1e-4 relative; bf16/f16 storage is exact in FP32, same bounds.
Singular vectors are compared after the sign convention, only where the
spectral gap exceeds 1e-3 of sigma_1."""

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


def _gap_ok(s, i, rel=1e-3):
    s = np.asarray(s)
    lo = s[i] - s[i + 1] if i + 1 < len(s) else s[i]
    hi = s[i - 1] - s[i] if i > 0 else np.inf
    return min(lo, hi) > rel * s[0]


def test_rsvd_small_fp64_matches_oracle(lib):
    """n=4096, m=256, sigma_i = exp(-i/10), p=4, l=128, k=20, seed 0.

    With l = 128 samples out of r = 1024 (with replacement, Sec. 2) two rows
    of this Omega repeat up to sign in every block, so range(B^T) has
    dimension 126.  Both sides take the rank-revealing basis of it (Q has 126
    columns, no arbitrary completion), which makes the rank-k result unique:
    U S V^T and S agree to 1e-12 relative, the singular vectors wherever the
    spectral gap is above 1e-3 sigma_1."""
    a, _ = synth.haar_spectrum(4096, 256, seed=1235)
    u, s, v = lib.bsrht_rsvd(torch.from_numpy(a).cuda(), 20, 128, 4, 0)
    torch.cuda.synchronize()
    u, s, v = u.cpu().numpy(), s.cpu().numpy(), v.cpu().numpy()
    ur, sr, vr = orl.rsvd(a, 20, 128, 4, 0)
    assert np.max(np.abs(s - sr)) <= 1e-12 * sr[0]
    for i in range(20):
        if _gap_ok(sr, i):
            assert np.linalg.norm(u[:, i] - ur[:, i]) <= 1e-10
            assert np.linalg.norm(v[:, i] - vr[:, i]) <= 1e-10
    approx = (u * s) @ v.T
    ref = (ur * sr) @ vr.T
    assert np.linalg.norm(approx - ref) <= 1e-12 * np.linalg.norm(ref)


def test_rsvd_rank_below_k_fp64(lib):
    """rank(A) = 5 < k = 8 < l = 16: range(B^T) has dimension 5, the output is
    the exact rank-5 factorization with zero trailing singular values and
    factor columns, as in the oracle."""
    a = synth.exact_rank(3000, 40, 5, seed=6)
    u, s, v = lib.bsrht_rsvd(torch.from_numpy(a).cuda(), 8, 16, 2, 1)
    torch.cuda.synchronize()
    u, s, v = u.cpu().numpy(), s.cpu().numpy(), v.cpu().numpy()
    ur, sr, vr = orl.rsvd(a, 8, 16, 2, 1)
    assert np.all(s[5:] == 0.0) and np.all(u[:, 5:] == 0.0) and np.all(v[:, 5:] == 0.0)
    np.testing.assert_allclose(s, sr, rtol=1e-12, atol=1e-13 * sr[0])
    assert np.linalg.norm(a - (u * s) @ v.T) <= 1e-12 * np.linalg.norm(a)


@pytest.mark.parametrize("p", [1, 4, 16])
def test_rsvd_exact_recovery_fp64(lib, p):
    a = synth.exact_rank(3000, 120, 20, seed=p)
    u, s, v = lib.bsrht_rsvd(torch.from_numpy(a).cuda(), 20, 40, p, 7)
    torch.cuda.synchronize()
    u, s, v = u.cpu().numpy(), s.cpu().numpy(), v.cpu().numpy()
    assert np.linalg.norm(a - (u * s) @ v.T) <= 1e-12 * np.linalg.norm(a)
    assert np.linalg.norm(u.T @ u - np.eye(20)) <= 1e-12
    assert np.linalg.norm(v.T @ v - np.eye(20)) <= 1e-12


def test_rsvd_fp64_beyond_65535_row_tiles(lib):
    """n = 2^22 + 4096 rows: the FP64 tall products (W = A Q and the tall QR)
    have more than 65535 row tiles of 64, which one grid dimension of the
    SIMT GEMM now carries; exact recovery of a rank-6 matrix as at small n."""
    n, m, r = (1 << 22) + 4096, 16, 6
    a = synth.exact_rank(n, m, r, seed=21)
    u, s, v = lib.bsrht_rsvd(torch.from_numpy(a).cuda(), r, 12, 4, 2)
    torch.cuda.synchronize()
    u, s, v = u.cpu().numpy(), s.cpu().numpy(), v.cpu().numpy()
    sv = np.linalg.svd(a, compute_uv=False)
    np.testing.assert_allclose(s, sv[:r], rtol=1e-12, atol=1e-13 * sv[0])
    assert np.linalg.norm(a - (u * s) @ v.T) <= 1e-12 * np.linalg.norm(a)
    assert np.linalg.norm(u.T @ u - np.eye(r)) <= 1e-12


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_rsvd_reduced_precision_matches_oracle(lib, dtype):
    a32 = synth.lowrank_noise(1 << 15, 384, rank=200, seed=12, dtype=np.float32)
    a_t = torch.from_numpy(a32).to(dtype)
    a64 = a_t.double().numpy()
    k, l, p = 30, 96, 4
    u, s, v = lib.bsrht_rsvd(a_t.cuda(), k, l, p, 3)
    torch.cuda.synchronize()
    u, s, v = u.cpu().numpy(), s.cpu().numpy(), v.cpu().numpy()
    ur, sr, vr = orl.rsvd(a64, k, l, p, 3)
    assert np.max(np.abs(s - sr)) <= 2e-5 * sr[0]
    err = np.linalg.norm(a64 - (u * s) @ v.T)
    err_ref = np.linalg.norm(a64 - (ur * sr) @ vr.T)
    assert abs(err - err_ref) <= 1e-4 * err_ref
    assert np.linalg.norm(u.T @ u - np.eye(k)) <= 1e-5
    assert np.linalg.norm(v.T @ v - np.eye(k)) <= 1e-5


def test_rsvd_ragged_and_edge_sizes(lib):
    """k = l = m (square sketch), odd sizes, p not dividing n."""
    a, _ = synth.haar_spectrum(1001, 37, seed=4)
    u, s, v = lib.bsrht_rsvd(torch.from_numpy(a).cuda(), 37, 37, 3, 1)
    torch.cuda.synchronize()
    u, s, v = u.cpu().numpy(), s.cpu().numpy(), v.cpu().numpy()
    sv = np.linalg.svd(a, compute_uv=False)
    np.testing.assert_allclose(s, sv, rtol=1e-10, atol=1e-12 * sv[0])
    assert np.linalg.norm(a - (u * s) @ v.T) <= 1e-10 * np.linalg.norm(a)


def test_rsvd_full_size_fp32_properties(lib):
    """n = 2^20, m = 4096, FP32, p = 4, l = 512, k = 100 in the benchmark's
    configuration. Properties that hold at any size: A V = U S exactly for
    Algorithm 1 (W = A Q = P R and R^T = U~ S~ V~^T), orthonormal factors,
    descending non-negative S."""
    n, m, k, l, p = 1 << 20, 4096, 100, 512, 4
    a = synth.lowrank_noise_device(n, m, seed=1236, dtype=torch.float32)
    u, s, v = lib.bsrht_rsvd(a, k, l, p, 0)
    torch.cuda.synchronize()
    av = torch.cat([(a[i:i + 65536].double() @ v) for i in range(0, n, 65536)])
    res = torch.linalg.norm(av - u * s) / torch.linalg.norm(s)
    assert res.item() <= 1e-4
    eye = torch.eye(k, device="cuda", dtype=torch.float64)
    assert torch.linalg.norm(u.T @ u - eye).item() <= 1e-4
    assert torch.linalg.norm(v.T @ v - eye).item() <= 1e-10
    sc = s.cpu().numpy()
    assert np.all(np.diff(sc) <= 0) and sc[-1] >= 0
    # The signal part has sigma_1 = 1 (i^-2 spectrum) plus the noise floor.
    assert 0.9 < sc[0] < 1.3


def _rbf(n, d, seed):
    x = synth.rbf_points(n, d, seed=seed).astype(np.float64)
    return synth.rbf_kernel(x, synth.rbf_bandwidth(x))


def test_nystrom_fp64_matches_oracle(lib):
    a = _rbf(1500, 20, 5)
    k, l, p = 40, 120, 4
    u, lam = lib.bsrht_nystrom(torch.from_numpy(a).cuda(), k, l, p, 2)
    torch.cuda.synchronize()
    u, lam = u.cpu().numpy(), lam.cpu().numpy()
    ur, lr, _ = orl.nystrom(a, k, l, p, 2)
    assert np.max(np.abs(lam - lr)) <= 1e-10 * lr[0]
    approx = (u * lam) @ u.T
    ref = (ur * lr) @ ur.T
    assert np.linalg.norm(approx - ref) <= 1e-9 * np.linalg.norm(a)


def test_nystrom_exact_recovery_fp64(lib):
    a = synth.psd_lowrank(2000, 15, seed=3)
    u, lam = lib.bsrht_nystrom(torch.from_numpy(a).cuda(), 15, 30, 4, 1)
    torch.cuda.synchronize()
    u, lam = u.cpu().numpy(), lam.cpu().numpy()
    assert np.linalg.norm(a - (u * lam) @ u.T) <= 1e-9 * np.linalg.norm(a)


def _fp32_eig_tol(n, lam1):
    """FP32 eigenvalue tolerance: the tall products (sketch, Z = Y C^-1, the Gram
    of Z) accumulate over up to n terms in FP32, so each computed eigenvalue
    of the rank-l Nystrom matrix carries an absolute error up to about
    8 sqrt(n) 2^-24 lambda_1; differences add with random signs over k."""
    return 8.0 * np.sqrt(n) * 2.0 ** -24 * lam1


@pytest.mark.parametrize("k", [100, 200, 400])
def test_nystrom_kernel_subsample_fp32(lib, k):
    """The kernel workload's 4096-point subsample (784-dim uniform points, RBF
    with the median bandwidth), p = 8, l = 600 (> r = 512, so Omega repeats
    rows and the core is singular): trace-norm error tr(A) - sum(Lambda), exact
    because the residual is PSD (Sec. 3.2), against the oracle run with the
    same FP32 rank threshold for Remark 3.1's SVD square root."""
    x = synth.rbf_points(4096, 784, seed=1238)
    h = synth.rbf_bandwidth(x)
    a64 = synth.rbf_kernel(x, h)
    a32 = a64.astype(np.float32)
    u, lam = lib.bsrht_nystrom(torch.from_numpy(a32).cuda(), k, 600, 8, 0)
    torch.cuda.synchronize()
    u, lam = u.cpu().numpy(), lam.cpu().numpy()
    ur, lr, _ = orl.nystrom(a32.astype(np.float64), k, 600, 8, 0, unit_roundoff=2.0 ** -23)
    tr = np.trace(a32.astype(np.float64))
    tol = _fp32_eig_tol(4096, lr[0])
    assert np.max(np.abs(lam - lr)) <= tol
    assert abs((tr - lam.sum()) - (tr - lr.sum())) <= np.sqrt(k) * tol
    assert np.linalg.norm(u.T @ u - np.eye(k)) <= 1e-4


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("p", [1, 8])
def test_nystrom_repeated_sketch_rows(lib, dtype, p):
    """l > sqrt(r): repeated rows of Omega make the core singular; both sides
    take Remark 3.1's SVD square root (same rank threshold) and agree on the
    eigenvalues and the trace error."""
    x = synth.rbf_points(2048, 16, seed=7).astype(np.float64)
    a = synth.rbf_kernel(x, synth.rbf_bandwidth(x))
    k, l, n = 150, 300, 2048
    u, lam = lib.bsrht_nystrom(torch.from_numpy(a).to(dtype).cuda(), k, l, p, 5)
    torch.cuda.synchronize()
    lam = lam.cpu().numpy()
    a_in = torch.from_numpy(a).to(dtype).double().numpy()
    ur_ = 2.0 ** -52 if dtype == torch.float64 else 2.0 ** -23
    _, lr, _ = orl.nystrom(a_in, k, l, p, 5, unit_roundoff=ur_)
    tr = np.trace(a_in)
    tol = 1e-10 * lr[0] if dtype == torch.float64 else _fp32_eig_tol(n, lr[0])
    assert np.max(np.abs(lam - lr)) <= tol
    assert abs((tr - lam.sum()) - (tr - lr.sum())) <= np.sqrt(k) * tol
