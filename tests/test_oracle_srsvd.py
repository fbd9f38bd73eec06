"""Pins of the oracle's single-view RSVD (Algorithm 3, Sec. 3.3) against what
fixes it from outside: exact recovery of a matrix of exact rank below l
(every step is then exact), the Eckart-Young lower bound and a loose
quasi-optimality bound on a decaying spectrum, orthonormal factors, and the
two-sided core sketch Phi A_p Psi^T being the same matrix in either
association order (the paper's definition fixes the product, not the
order)."""

import numpy as np
import pytest

from oracle import bsrht as ob
from oracle import lowrank as orl
import synth


@pytest.mark.parametrize("n,m,r,k,l,s,p,seed", [
    (512, 64, 10, 10, 20, 40, 4, 7),
    (1000, 96, 12, 8, 24, 48, 3, 1),
    (256, 256, 20, 20, 40, 64, 1, 2),
])
def test_exact_recovery(n, m, r, k, l, s, p, seed):
    a = synth.exact_rank(n, m, r, seed=seed + 10)
    u, sv, v = orl.srsvd(a, k, l, s, p, seed)
    if k == r:
        assert np.linalg.norm(a - (u * sv) @ v.T) <= 1e-12 * np.linalg.norm(a)
    ref = np.linalg.svd(a, compute_uv=False)[:k]
    np.testing.assert_allclose(sv, ref, rtol=1e-10, atol=1e-12 * ref[0])


@pytest.mark.parametrize("k,l,s", [(10, 40, 80), (20, 60, 120)])
def test_quasi_optimality(k, l, s):
    a, sig = synth.haar_spectrum(2048, 128, seed=5)
    opt = np.sqrt(np.sum(np.asarray(sig, dtype=np.float64)[k:] ** 2))
    for seed in range(3):
        u, sv, v = orl.srsvd(a, k, l, s, 4, seed)
        err = np.linalg.norm(a - (u * sv) @ v.T)
        assert opt * (1 - 1e-12) <= err <= 2.0 * opt
        assert np.linalg.norm(u.T @ u - np.eye(k)) <= 1e-12
        assert np.linalg.norm(v.T @ v - np.eye(k)) <= 1e-12
        assert np.all(np.diff(sv) <= 0) and sv[-1] >= 0


def test_core_sketch_association():
    """Z^T = Psi (A Phi^T) computed as in the algorithm equals
    (Phi (Psi A)^T)^T, the other association order."""
    rng = np.random.default_rng(3)
    a = rng.standard_normal((300, 40))
    seeds = orl.srsvd_seeds(5)
    s, p = 24, 3
    w = ob.sketch_dense(a.T, 1, s, seeds[2]).T           # A Phi^T (n x s)
    zt = ob.sketch_dense(w, p, s, seeds[3])             # Psi A Phi^T (s x s)
    v = ob.sketch_dense(a, p, s, seeds[3])               # Psi A (s x m)
    zt2 = ob.sketch_dense(v.T, 1, s, seeds[2]).T         # (Phi (Psi A)^T)^T
    np.testing.assert_allclose(zt, zt2, rtol=0, atol=1e-12 * np.abs(zt).max())


def test_seeds_are_distinct():
    assert len(set(orl.srsvd_seeds(2**64 - 2))) == 4
    assert orl.srsvd_seeds(2**64 - 1)[1] == 0
