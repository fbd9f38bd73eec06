"""Matrix-free Nystrom (bsrht_nystrom_rbf): Algorithm 2 on the RBF kernel
matrix A_ij = exp(-|x_i - x_j|^2 / (2 h^2)) of a point set, with A formed a
column panel at a time and sketched right away (never stored).

Against the CPU oracle on the kernel workload's 4096-point subsample (784
dimensions, median bandwidth), with the FP32 tolerances of the stored-matrix
test (tests/test_gpu_lowrank.py): the entries of A differ from the oracle's
FP64 matrix by FP32 rounding on both paths.  Against the stored-matrix path
on a larger point set whose panels do not divide n."""

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


def _fp32_eig_tol(n, lam1):
    """As in test_gpu_lowrank: FP32 tall products over up to n terms."""
    return 8.0 * np.sqrt(n) * 2.0 ** -24 * lam1


@pytest.mark.parametrize("k", [100, 400])
def test_rbf_nystrom_subsample_matches_oracle(lib, k):
    x = synth.rbf_points(4096, 784, seed=1238)
    h = synth.rbf_bandwidth(x)
    a64 = synth.rbf_kernel(x, h)
    u, lam = lib.bsrht_nystrom_rbf(torch.from_numpy(x).cuda(), h, k, 600, 8, 0)
    torch.cuda.synchronize()
    u, lam = u.cpu().numpy(), lam.cpu().numpy()
    _, lr, _ = orl.nystrom(a64, k, 600, 8, 0, unit_roundoff=2.0 ** -23)
    tr = np.trace(a64)
    tol = _fp32_eig_tol(4096, lr[0])
    assert np.max(np.abs(lam - lr)) <= tol
    assert abs((tr - lam.sum()) - (tr - lr.sum())) <= np.sqrt(k) * tol
    assert np.linalg.norm(u.T @ u - np.eye(k)) <= 1e-4


def test_rbf_nystrom_matches_stored_matrix_ragged_panels(lib):
    """n = 40000 points in 16 dimensions: panels of 6656 columns (the last
    one narrower); the stored FP32 matrix from the same points through
    bsrht_nystrom gives the same eigenvalues to FP32 accuracy."""
    n, dim, k, l, p = 40000, 16, 50, 200, 4
    x = torch.from_numpy(synth.rbf_points(n, dim, seed=21)).cuda()
    h = synth.rbf_bandwidth(x.cpu().numpy())
    a = synth.rbf_kernel_device(x, h, dtype=torch.float32)
    _, lam_s = lib.bsrht_nystrom(a, k, l, p, 3)
    del a
    torch.cuda.empty_cache()
    _, lam_f = lib.bsrht_nystrom_rbf(x, h, k, l, p, 3)
    torch.cuda.synchronize()
    lam_s, lam_f = lam_s.cpu().numpy(), lam_f.cpu().numpy()
    assert np.max(np.abs(lam_f - lam_s)) <= _fp32_eig_tol(n, lam_s[0])


def test_rbf_nystrom_rejects(lib):
    x = torch.zeros(256, 8, device="cuda", dtype=torch.float32)
    with pytest.raises(lib.BsrhtError) as e:
        lib.bsrht_nystrom_rbf(x, 0.0, 4, 8, 2, 0)  # h = 0
    assert e.value.status == -22
    with pytest.raises(lib.BsrhtError) as e:
        lib.bsrht_nystrom_rbf(torch.zeros(256, 6, device="cuda", dtype=torch.float32), 1.0, 4, 8, 2, 0)  # dim % 4
    assert e.value.status == -95
    with pytest.raises(lib.BsrhtError) as e:
        lib.bsrht_nystrom_rbf(x, 1.0, 9, 8, 2, 0)  # k > l
    assert e.value.status == -22
