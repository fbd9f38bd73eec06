"""Pins of the CPU oracle's randomized SVD (Algorithm 1) and Nystrom
(Algorithm 2) against closed forms, LAPACK special cases and the bounds of
Sec. 3 (no GPU)."""

import math

import numpy as np
import pytest

from oracle import bsrht, lowrank
import synth


def test_sign_normalize():
    u = np.array([[1.0, -3.0], [-2.0, 1.0]])
    v = np.array([[1.0, 1.0]])
    un, vn = lowrank.sign_normalize(u, v)
    assert np.array_equal(un, [[-1.0, 3.0], [2.0, -1.0]])
    assert np.array_equal(vn, [[-1.0, -1.0]])


def test_best_rank_k_errors_closed_form():
    """Sec. 3: spectral sigma_{k+1}, trace sum of the tail, Frobenius norm of the tail."""
    s = np.array([5.0, 4.0, 3.0, 2.0, 1.0])
    e = lowrank.best_rank_k_errors(s, 2)
    assert e == {"spectral": 3.0, "trace": 6.0, "fro": math.sqrt(14.0)}
    a, _ = synth.haar_spectrum(200, 40, seed=1)
    u, sk, v = lowrank.truncated_svd(a, 5)
    sv = np.linalg.svd(a, compute_uv=False)
    assert abs(np.linalg.norm(a - (u * sk) @ v.T, 2) - sv[5]) < 1e-12


@pytest.mark.parametrize("p", [1, 4, 8])
def test_rsvd_exact_recovery(p):
    """range(A Omega^T) captures an exact rank-r matrix when r < l (w.p. 1)."""
    a = synth.exact_rank(600, 80, 20, seed=3)
    u, s, v = lowrank.rsvd(a, 20, 32, p, seed=5)
    assert np.linalg.norm(a - (u * s) @ v.T) <= 1e-12 * np.linalg.norm(a)
    np.testing.assert_allclose(s, 1.0 / np.arange(1, 21), rtol=1e-12)


def test_rsvd_full_sketch_is_truncated_svd():
    """With l = m the sketch spans all of R^m, so Algorithm 1 returns the
    truncated SVD that LAPACK computes directly (Eckart-Young optimum)."""
    a, _ = synth.haar_spectrum(512, 32, seed=2)
    u, s, v = lowrank.rsvd(a, 8, 32, 4, seed=1)
    ur, sr, vr = lowrank.truncated_svd(a, 8)
    np.testing.assert_allclose(s, sr, rtol=1e-12)
    np.testing.assert_allclose(u, ur, atol=1e-10)
    np.testing.assert_allclose(v, vr, atol=1e-10)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rsvd_eckart_young_and_quasi_optimality(seed):
    """Errors are >= the Eckart-Young optimum and <= opt + 2.5 ||A - [[A]]_d||_F
    (the RSVD bound of Sec. 3.1 with d = l/4)."""
    a, sig = synth.haar_spectrum(2048, 128, seed=11)
    k, l = 10, 64
    u, s, v = lowrank.rsvd(a, k, l, 4, seed)
    res = a - (u * s) @ v.T
    opt = lowrank.best_rank_k_errors(sig, k)
    tail_d = lowrank.best_rank_k_errors(sig, l // 4)["fro"]
    fro = np.linalg.norm(res)
    spec = np.linalg.norm(res, 2)
    assert fro >= opt["fro"] * (1 - 1e-12)
    assert spec >= opt["spectral"] * (1 - 1e-12)
    assert fro <= opt["fro"] + 2.5 * tail_d
    assert spec <= opt["spectral"] + 2.5 * tail_d
    # Orthonormal factors
    assert np.linalg.norm(u.T @ u - np.eye(k)) < 1e-12
    assert np.linalg.norm(v.T @ v - np.eye(k)) < 1e-12


def test_nystrom_exact_recovery():
    """A PSD matrix of exact rank r < l is reproduced (up to the shift)."""
    a = synth.psd_lowrank(400, 15, seed=2)
    u, lam, nu = lowrank.nystrom(a, 15, 30, 4, seed=3)
    assert nu > 0
    assert np.linalg.norm(a - (u * lam) @ u.T) <= 1e-9 * np.linalg.norm(a)
    np.testing.assert_allclose(lam, 1.0 / np.arange(1, 16), rtol=1e-8)


def test_nystrom_algorithm_matches_definition():
    """Algorithm 2 with k = l equals the Nystrom matrix of Sec. 3.2,
    (Omega A)^T (Omega A Omega^T)^+ (Omega A), up to the O(nu) shift."""
    x = synth.rbf_points(300, 6, seed=4).astype(np.float64)
    h = synth.rbf_bandwidth(x)
    a = synth.rbf_kernel(x, h)
    l = 40
    u, lam, nu = lowrank.nystrom(a, l, l, 4, seed=8)
    ref = lowrank.nystrom_full(a, l, 4, seed=8)
    assert np.linalg.norm((u * lam) @ u.T - ref) <= 1e-7 * np.linalg.norm(a)


def test_nystrom_repeated_sketch_rows_matches_definition():
    """l > r makes R sample the same row repeatedly; with few blocks some rows
    of Omega repeat up to sign and the core is singular even after the shift.
    Remark 3.1's SVD square root then reproduces the pseudo-inverse definition
    of Sec. 3.2."""
    x = synth.rbf_points(256, 6, seed=9).astype(np.float64)
    a = synth.rbf_kernel(x, synth.rbf_bandwidth(x))
    l, p = 48, 8  # r = 32 < l
    om = bsrht.dense_omega(256, p, l, 3)
    assert np.linalg.matrix_rank(om) < l
    u, lam, nu = lowrank.nystrom(a, l, l, p, seed=3)
    ref = lowrank.nystrom_full(a, l, p, seed=3)
    assert np.linalg.norm((u * lam) @ u.T - ref) <= 1e-7 * np.linalg.norm(a)


def test_nystrom_residual_is_psd_and_trace_identity():
    """Sec. 3.2: A - [[A]]^(Nyst) is PSD, so its trace norm is tr(A) - tr(A^)."""
    x = synth.rbf_points(256, 5, seed=5).astype(np.float64)
    a = synth.rbf_kernel(x, synth.rbf_bandwidth(x))
    ah = lowrank.nystrom_full(a, 32, 4, seed=1)
    res = a - ah
    ev = np.linalg.eigvalsh(0.5 * (res + res.T))
    assert ev.min() >= -1e-9 * np.trace(a)
    assert abs(np.sum(np.abs(ev)) - (np.trace(a) - np.trace(ah))) <= 1e-8 * np.trace(a)


@pytest.mark.parametrize("seed", [0, 1])
def test_nystrom_trace_bounds(seed):
    """Eckart-Young lower bound and the Nystrom bound of Sec. 3.2,
    ||A - [[A]]_k^(Nyst)||_* <= ||A - [[A]]_k||_* + 3 ||A - [[A]]_d||_*."""
    x = synth.rbf_points(512, 8, seed=6).astype(np.float64)
    a = synth.rbf_kernel(x, 0.5 * synth.rbf_bandwidth(x))
    lam_all = np.linalg.eigvalsh(a)[::-1]
    k, l = 20, 80
    u, lam, _ = lowrank.nystrom(a, k, l, 4, seed)
    res = a - (u * lam) @ u.T
    trace_err = np.sum(np.abs(np.linalg.eigvalsh(0.5 * (res + res.T))))
    opt = np.sum(lam_all[k:])
    tail_d = np.sum(lam_all[l // 4:])
    assert trace_err >= opt * (1 - 1e-10)
    assert trace_err <= opt + 3 * tail_d


def test_nystrom_shift_rule():
    """Remark 3.1 reading: nu = sqrt(n) eps ||Y||_F."""
    y = np.ones((16, 3))
    assert lowrank.nystrom_shift(y) == 4.0 * 2.0 ** -52 * math.sqrt(48.0)


# ---- rank-revealing basis of range(Y) (Algorithm 1 step 2) -------------------

def _independent_row_classes(n, p, l, seed):
    """Rows of Omega grouped by linear dependence, from the eq. 2.3 definition
    alone: row j of block i is Dt^(i)_jj H_r[s_j, :] D^(i) / sqrt(l), so rows
    j and j' are parallel exactly when s_j = s_j' and the sign ratio
    Dt^(i)_jj / Dt^(i)_j'j' is the same in every block (Hadamard rows with
    different s are orthogonal)."""
    rb, r = bsrht.block_layout(n, p)
    s = bsrht.samples(seed, l, r)
    dts = np.array([bsrht.dt_signs(seed, i, l) for i in range(p)])  # p x l
    classes = {}
    for j in range(l):
        pat = tuple(dts[:, j] * dts[0, j])
        classes.setdefault((int(s[j]), pat), []).append(j)
    return list(classes.values())


def test_range_basis_rank_of_config1_sketch():
    """n = 4096, m = 256, p = 4, l = 128, seed 0: two pairs of rows of Omega
    are parallel, so range(Y) has dimension 126 and Q has 126 columns."""
    a, _ = synth.haar_spectrum(4096, 256, seed=1235)
    cls = _independent_row_classes(4096, 4, 128, 0)
    assert len(cls) == 126
    y = bsrht.sketch_dense(a, 4, 128, 0).T
    q = lowrank.range_basis(y)
    assert q.shape == (256, 126)
    assert np.linalg.norm(q.T @ q - np.eye(126)) <= 1e-13
    # Q spans range(Y): projecting Y onto it leaves rounding only.
    assert np.linalg.norm(y - q @ (q.T @ y)) <= 1e-14 * np.linalg.norm(y)


@pytest.mark.parametrize("n,m,p,l,seed,k", [(4096, 256, 4, 128, 0, 20), (512, 96, 1, 48, 3, 10)])
def test_rsvd_repeated_rows_is_truncated_svd_of_projection(n, m, p, l, seed, k):
    """With parallel rows in Omega the output of Algorithm 1 is the truncated
    SVD of A Pi, Pi the orthogonal projector onto range(A^T Omega^T) (the
    paper's range(Y)).  Pi is built here without the oracle's basis: from one
    representative row per class of parallel rows (full row rank), by
    Householder QR of A^T Omega_d^T."""
    if n == 4096:
        a, _ = synth.haar_spectrum(n, m, seed=1235)
    else:
        a = synth.gaussian(n, m, seed=4)
    cls = _independent_row_classes(n, p, l, seed)
    assert len(cls) < l
    om = bsrht.dense_omega(n, p, l, seed)
    om_d = om[[c[0] for c in cls]]
    qd, _ = np.linalg.qr(a.T @ om_d.T)
    ap = a @ qd @ qd.T
    ur, sr, vr = lowrank.truncated_svd(ap, k)
    u, s, v = lowrank.rsvd(a, k, l, p, seed)
    np.testing.assert_allclose(s, sr, rtol=1e-12, atol=1e-13 * sr[0])
    ref = (ur * sr) @ vr.T
    assert np.linalg.norm((u * s) @ v.T - ref) <= 1e-12 * np.linalg.norm(ref)


def test_range_basis_rule_is_relative_and_scale_free():
    """Directions with sigma <= l 2^-44 sigma_1 are dropped, larger ones kept,
    whatever the scale of Y: sigma ratios 1, 1e-3, 1e-11 (kept) and 1e-14
    and an exact null direction (dropped), scaled by 1e-150 and 1e150."""
    rng = np.random.default_rng(2)
    u = np.linalg.qr(rng.standard_normal((40, 5)))[0]
    v = np.linalg.qr(rng.standard_normal((5, 5)))[0]
    for scale in (1e-150, 1.0, 1e150):
        y = (u * (scale * np.array([1.0, 1e-3, 1e-11, 1e-14, 0.0]))) @ v.T
        q = lowrank.range_basis(y)
        assert q.shape == (40, 3)
        p_ref = u[:, :3] @ u[:, :3].T
        assert np.linalg.norm(q @ q.T - p_ref) <= 1e-4  # the 1e-11 direction is resolved to ~1e-5
    assert lowrank.range_tol(128) == 128 * 2.0 ** -44


def test_rsvd_rank_below_k_pads_with_zeros():
    """If range(Y) has dimension r' < k, the rank-k output is the rank-r'
    approximation: trailing singular values and factor columns are zero."""
    a = synth.exact_rank(300, 40, 5, seed=6)
    u, s, v = lowrank.rsvd(a, 8, 16, 2, seed=1)
    assert np.all(s[5:] == 0.0) and np.all(u[:, 5:] == 0.0) and np.all(v[:, 5:] == 0.0)
    assert np.linalg.norm(a - (u * s) @ v.T) <= 1e-12 * np.linalg.norm(a)


# ---- Remark 3.1's rank threshold of the Nystrom core ------------------------

def _core(lams, seed=0):
    rng = np.random.default_rng(seed)
    v = np.linalg.qr(rng.standard_normal((len(lams), len(lams))))[0]
    c = (v * np.asarray(lams)) @ v.T
    return 0.5 * (c + c.T), v


def test_nystrom_core_factor_cholesky_when_well_conditioned():
    core, _ = _core([4.0, 2.0, 1.0, 0.5, 0.25])
    f, r = lowrank.nystrom_core_factor(core, 5)
    assert r == 5
    assert np.allclose(np.triu(np.linalg.inv(f)), np.linalg.inv(f))  # F = C^-1, C upper
    np.testing.assert_allclose(f @ f.T, np.linalg.inv(core), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("u,expect_rank", [(2.0 ** -52, 6), (2.0 ** -23, 5)])
def test_nystrom_core_factor_threshold_is_l_times_unit_roundoff(u, expect_rank):
    """tau = l u: an eigenvalue ratio of 1e-9 lies above l 2^-52 (kept, the
    Cholesky path) and below l 2^-23 (dropped by the SVD square root)."""
    lams = [1.0, 0.7, 0.3, 0.1, 0.05, 1e-9]
    core, v = _core(lams, seed=1)
    f, r = lowrank.nystrom_core_factor(core, 6, unit_roundoff=u)
    assert r == expect_rank
    keep = np.array(lams) > 6 * u
    pinv = (v[:, keep] / np.array(lams)[keep]) @ v[:, keep].T
    assert np.linalg.norm(f @ f.T - pinv) <= 1e-6 * np.linalg.norm(pinv)


def test_nystrom_core_factor_exactly_singular_core():
    """A core of exact rank 3 (l = 5): the SVD square root keeps 3 directions
    and F F^T is the pseudo-inverse."""
    core, v = _core([3.0, 2.0, 1.0, 0.0, 0.0], seed=2)
    f, r = lowrank.nystrom_core_factor(core, 5)
    assert r == 3
    assert np.all(f[:, 3:] == 0.0)
    np.testing.assert_allclose(f @ f.T, np.linalg.pinv(core, hermitian=True, rcond=1e-12), atol=1e-10)
