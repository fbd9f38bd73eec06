"""Randomized SVD (Algorithm 1) and randomized Nystrom (Algorithm 2) on the
block SRHT sketch, plain FP64 numpy/LAPACK. TEST INFRASTRUCTURE ONLY.

Orientation. The paper states both algorithms for an m x n matrix with m <= n
and the sketch Y = A Omega^T. This library takes the tall n x m matrix (the
paper's A transposed) and forms B = Omega A, so the paper's Y is B^T here and
the roles of the two factors swap (Sec. 3.1, Algorithm 1, last step):
U = P V~_k, S = Sigma~_k, V = Q U~_k.

Readings of the paper used here (each also listed with the design notes):

* Algorithm 1, step 2: Q is an orthonormal basis of range(Y) (Sec. 3.1).
  Sampling with replacement (Sec. 2) lets Omega repeat a row up to sign in
  every block, and then range(Y) has dimension r' < l; completing Q with
  arbitrary directions would make the result depend on them. Q is therefore
  rank revealing: the left singular vectors of Y (LAPACK SVD) whose singular
  value exceeds tau * sigma_1, tau = l * 2^-44 (see range_tol). Steps 3-6
  then run on r' columns; with r' < k the trailing singular values and the matching columns
  of U and V are zero. Step 4 uses Householder QR (LAPACK geqrf/orgqr via
  numpy) and step 5 the SVD of the small R^T factor (LAPACK gesdd).
* Algorithm 2, step 6 writes (Y V~_k) Sigma~_k^-1; with Z = Q~ R and
  R = U~ Sigma~ V~^T the quantity that equals Q~ U~_k (the stabler variant
  the text mentions) is (Z V~_k) Sigma~_k^-1, so Z is used.
* Remark 3.1 only says "shift as in Li et al."; the shift used is
  nu = sqrt(n) * 2^-52 * ||Y||_F, Y_nu = Y + nu Omega^T,
  core = sym(Omega Y_nu), Lambda = max(Sigma~_k^2 - nu, 0). The shift does not
  help when Omega itself has repeated rows (sampling with replacement allows
  them), so when the Cholesky factorisation fails or its squared pivots fall
  below tau = l * u of the largest (u the unit roundoff of the arithmetic of
  A's tall products: 2^-52 for FP64 data, 2^-23 otherwise), Remark 3.1's
  other remedy is used: the SVD square root of the core, as a pseudo-inverse
  (eigenvalues below tau * lambda_max dropped).
* Cholesky convention: C upper triangular with C^T C = core, Z = Y C^-1.
* Singular vectors are only defined up to sign: each column of U is flipped
  so its largest-magnitude entry (lowest index on ties) is positive, and the
  matching column of V gets the same flip.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla

from .bsrht import dense_omega, sketch_dense
from .gaussian import gaussian_sketch, omega_gaussian

EPS64 = 2.0 ** -52


def sign_normalize(u: np.ndarray, v: np.ndarray | None = None):
    """Flip columns so that each column's largest-|.| entry is positive."""
    u = np.array(u, copy=True)
    idx = np.argmax(np.abs(u), axis=0)
    sg = np.sign(u[idx, np.arange(u.shape[1])])
    sg[sg == 0] = 1.0
    u *= sg
    if v is None:
        return u
    v = np.array(v, copy=True) * sg
    return u, v


def best_rank_k_errors(sigma: np.ndarray, k: int) -> dict:
    """Eckart-Young optimal errors of a rank-k approximation (Sec. 3):
    spectral sigma_{k+1}, trace sum_{i>k} sigma_i, Frobenius (sum sigma_i^2)^1/2."""
    tail = np.asarray(sigma, dtype=np.float64)[k:]
    return {
        "spectral": float(tail[0]) if tail.size else 0.0,
        "trace": float(np.sum(tail)),
        "fro": float(math.sqrt(np.sum(tail * tail))),
    }


def truncated_svd(a: np.ndarray, k: int):
    """Best rank-k approximation [[A]]_k by LAPACK SVD: (U_k, s_k, V_k)."""
    u, s, vt = np.linalg.svd(np.asarray(a, dtype=np.float64), full_matrices=False)
    uk, vk = sign_normalize(u[:, :k], vt[:k].T)
    return uk, s[:k], vk


# Relative precision the FP64 sketch is computed to: its Walsh-Hadamard
# transform is exact on fixed-point values with at least 45 fraction bits
# below each column's largest magnitude; 2^-44 bounds that conversion.
SKETCH_PRECISION = 2.0 ** -44


def range_tol(l: int) -> float:
    """Rank rule of the basis of range(Y): directions with sigma <= tau sigma_1
    are numerically absent, tau = l * 2^-44 (l columns times the relative
    precision of the FP64 sketch), so that directions that are zero in exact
    arithmetic are dropped whatever rounding the sketch carried."""
    return l * SKETCH_PRECISION


def range_basis(y: np.ndarray) -> np.ndarray:
    """Orthonormal basis of the numerical range of y (rows x l): the left
    singular vectors (LAPACK SVD) with sigma_i > range_tol(l) * sigma_1.
    Returns a rows x r' matrix, r' <= l (r' = 0 for y = 0)."""
    y = np.asarray(y, dtype=np.float64)
    if y.shape[1] == 0:
        return np.zeros((y.shape[0], 0))
    u, s, _ = np.linalg.svd(y, full_matrices=False)
    if s[0] == 0.0:
        return np.zeros((y.shape[0], 0))
    keep = s > range_tol(y.shape[1]) * s[0]
    return np.ascontiguousarray(u[:, keep])


def rsvd(a: np.ndarray, k: int, l: int, p: int, seed: int, sketch: str = "bsrht"):
    """Algorithm 1 for the tall n x m matrix ``a``; returns (U n x k, S k, V m x k).
    ``sketch="gaussian"`` takes Omega from ``oracle.gaussian`` (the comparator
    of Sec. 4; p is then unused)."""
    a = np.asarray(a, dtype=np.float64)
    n, m = a.shape
    # Step 1: Y = A_paper Omega^T = (Omega A)^T, m x l.
    if sketch == "gaussian":
        y = gaussian_sketch(a, l, seed).T
    else:
        y = sketch_dense(a, p, l, seed).T
    # Step 2: orthonormal basis Q of range(Y), rank revealing (m x r').
    q = range_basis(y)
    r = q.shape[1]
    # Step 3: Z = Q^T A_paper = (A Q)^T; step 4 needs Z^T = A Q = P R.
    zt = a @ q
    pmat, rmat = np.linalg.qr(zt)
    # Step 5: SVD of R^T (r' x r'), truncated to rank k.
    ut, st, vtt = np.linalg.svd(rmat.T)
    # Step 6: A_paper ~ (Q U~_k) S~_k (P V~_k)^T, so A ~ (P V~_k) S~_k (Q U~_k)^T.
    kk = min(k, r)
    u = np.zeros((n, k))
    v = np.zeros((m, k))
    s = np.zeros(k)
    u[:, :kk] = pmat @ vtt[:kk].T
    v[:, :kk] = q @ ut[:, :kk]
    s[:kk] = st[:kk]
    u, v = sign_normalize(u, v)
    return u, s, v


def srsvd_seeds(seed: int):
    """Seeds of Omega, Gamma, Phi, Psi in the single-view RSVD: seed + 0..3
    (mod 2^64); one key per sketching matrix of the same generator."""
    return tuple((seed + i) & ((1 << 64) - 1) for i in range(4))


def srsvd(a: np.ndarray, k: int, l: int, s: int, p: int, seed: int):
    """Single-view RSVD, Algorithm 3 of Sec. 3.3, for the tall n x m matrix
    ``a`` (the paper's m x n matrix is a^T); returns (U n x k, S k, V m x k).

    Sketching matrices, seeds from ``srsvd_seeds``: Omega (l x n, p blocks),
    Phi (s x m, one block) and Psi (s x n, p blocks) are block SRHTs (eq. 2.3);
    Gamma (l x m) is the Gaussian map of ``oracle.gaussian`` (an SRHT row
    sample of l out of r ~ m repeats rows, which would make X rank deficient;
    Algorithm 3 takes any oblivious embedding).  In the paper's notation
    (A_p = a^T): X = A_p^T Gamma^T, Y = A_p Omega^T, Z = Phi A_p Psi^T;
    Q = orth(Y) (m x rq), P = orth(X) (n x rp), both rank revealing
    (``range_basis``); C = (Phi Q)^+ Z ((Psi P)^T)^+
    (the reading of step 4: pseudo-inverses by least squares, the right one
    applied to (Psi P)^T so that the product is defined); C = U~ S~ V~^T;
    A_p ~ (Q U~_k) S~_k (P V~_k)^T, i.e. a ~ (P V~_k) S~_k (Q U~_k)^T.
    """
    a = np.asarray(a, dtype=np.float64)
    s_om, s_ga, s_ph, s_ps = srsvd_seeds(seed)
    # Step 1: the three sketches (each a linear function of a alone).
    y = sketch_dense(a, p, l, s_om).T              # m x l = A_p Omega^T
    x = a @ omega_gaussian(a.shape[1], l, s_ga).T  # n x l = A_p^T Gamma^T
    w = sketch_dense(a.T, 1, s, s_ph).T            # n x s = a Phi^T
    z = sketch_dense(w, p, s, s_ps).T              # s x s = Phi A_p Psi^T
    # Step 2: orthonormal bases, rank revealing as in Algorithm 1
    # (range_basis): Q is m x rq, P is n x rp.
    q = range_basis(y)
    pm = range_basis(x)
    # Step 3: Phi Q (s x rq) and Psi P (s x rp).
    phq = sketch_dense(q, 1, s, s_ph)
    psp = sketch_dense(pm, p, s, s_ps)
    # Step 4: C = (Phi Q)^+ Z ((Psi P)^T)^+ by least squares (rq x rp).
    c1 = np.linalg.lstsq(phq, z, rcond=None)[0]    # rq x s
    c = np.linalg.lstsq(psp, c1.T, rcond=None)[0].T  # rq x rp
    # Step 5: SVD of C; step 6: the factors (zero beyond the numerical rank).
    uc, sc, vct = np.linalg.svd(c)
    n, m = a.shape
    kk = min(k, sc.size)
    u = np.zeros((n, k))
    v = np.zeros((m, k))
    sv = np.zeros(k)
    u[:, :kk] = pm @ vct[:kk].T
    v[:, :kk] = q @ uc[:, :kk]
    sv[:kk] = sc[:kk]
    u, v = sign_normalize(u, v)
    return u, sv, v


def nystrom_shift(y: np.ndarray) -> float:
    """nu = sqrt(n) * eps * ||Y||_F (reading of Remark 3.1)."""
    return math.sqrt(y.shape[0]) * EPS64 * float(np.linalg.norm(y))


def nystrom_core_factor(core: np.ndarray, l: int, unit_roundoff: float = EPS64):
    """Right factor F of Algorithm 2 step 3 (Z = Y_nu F) and its rank.

    Step 2 takes the Cholesky factor C (upper, C^T C = core) and F = C^-1.
    Remark 3.1: when the core is numerically rank deficient -- the
    factorization fails, or its squared pivots fall below tau times the
    largest -- F is the SVD square root's pseudo-inverse V_r lambda_r^-1/2
    (eigenvalues lambda <= tau lambda_max dropped, the columns of the dropped
    directions zero).  tau = l * unit_roundoff, the unit roundoff of the
    arithmetic of the tall products (2^-52 for FP64 data, 2^-23 for FP32 and
    16-bit data).  Returns (F l x l, rank)."""
    tau = l * unit_roundoff
    try:
        c = sla.cholesky(core, lower=False)
        piv = np.diag(c) ** 2
        if piv.min() > tau * piv.max():
            return sla.solve_triangular(c, np.eye(l), lower=False), l
    except np.linalg.LinAlgError:
        pass
    lam_c, v_c = np.linalg.eigh(core)
    lam_c, v_c = lam_c[::-1], v_c[:, ::-1]   # descending
    keep = lam_c > tau * lam_c[0]
    r = int(keep.sum())
    f = np.zeros((l, l))
    f[:, :r] = v_c[:, :r] / np.sqrt(lam_c[:r])
    return f, r


def nystrom(a: np.ndarray, k: int, l: int, p: int, seed: int, shift: bool = True,
            unit_roundoff: float = EPS64):
    """Algorithm 2 (with the Z fix in step 6 and the remedies of Remark 3.1).

    ``a`` is n x n symmetric PSD. Returns (U n x k, Lambda k, nu) with
    A ~ U diag(Lambda) U^T. ``unit_roundoff`` is the unit roundoff of the
    arithmetic of A's tall products (2^-52 for FP64 data, 2^-23 for FP32 and
    16-bit data, as on the device): it sets the rank threshold
    tau = l * unit_roundoff of Remark 3.1's SVD square root
    (``nystrom_core_factor``).
    """
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[0]
    om = dense_omega(n, p, l, seed)
    # Step 1: Y = A Omega^T (n x l), shifted: Y_nu = Y + nu Omega^T.
    y = a @ om.T
    nu = nystrom_shift(y) if shift else 0.0
    y_nu = y + nu * om.T
    core = om @ y_nu
    core = 0.5 * (core + core.T)
    # Steps 2-3: Z = Y_nu F with F = C^-1 (Cholesky) or Remark 3.1's SVD
    # square root (see nystrom_core_factor).
    f, _ = nystrom_core_factor(core, l, unit_roundoff)
    z = y_nu @ f
    # Step 4: R factor of Z.
    rmat = np.linalg.qr(z, mode="r")
    # Step 5: SVD of R.
    _, sr, vrt = np.linalg.svd(rmat)
    # Step 6: U^ = (Z V~_k) Sigma~_k^-1.
    sk = sr[:k]
    u = np.divide(z @ vrt[:k].T, sk, out=np.zeros((z.shape[0], k)), where=sk > 0)
    # Step 7: A ~ U^ Sigma~_k^2 U^^T, minus the shift.
    lam = np.maximum(sr[:k] ** 2 - nu, 0.0)
    u = sign_normalize(u)
    return u, lam, nu


def nystrom_full(a: np.ndarray, l: int, p: int, seed: int) -> np.ndarray:
    """The untruncated Nystrom matrix (Omega A)^T (Omega A Omega^T)^+ (Omega A)
    by its definition in Sec. 3.2 (pseudo-inverse, no shift)."""
    a = np.asarray(a, dtype=np.float64)
    om = dense_omega(a.shape[0], p, l, seed)
    b = om @ a
    core = b @ om.T
    return b.T @ np.linalg.pinv(core, hermitian=True) @ b
