"""Seeded synthetic inputs shaped like the workloads of the block-SRHT paper.

This module only draws test matrices. It holds none of the sketching or
low-rank arithmetic: both the CUDA path and the CPU oracle receive the bytes
produced here, so the two sides see identical inputs.

Workloads (the paper's own datasets, MNIST and YearPredictionMSD in Sec. 4.1,
are not available here; these seeded stand-ins keep their shapes and the
spectral structure the experiments rely on):

* ``haar_spectrum``     A = U diag(sigma) V^T with Haar-random U, V and
                        sigma_i = exp(-i/10)   (small FP64 case, n=4096, m=256).
* ``lowrank_noise``     A = G1 diag(i^-2) G2^T + 1e-4 N with orthonormalised
                        Gaussian factors of rank 1000 (tall-skinny case of
                        Sec. 4.2, n up to 2^20).
* ``rbf_points`` / ``rbf_kernel``  x_i ~ U[0,1]^784, A_ij = exp(-|xi-xj|^2/(2h^2)),
                        h = median pairwise distance of a seeded 4096-point
                        subsample (the kernel-matrix case of Sec. 4.1).
* ``gaussian``          plain i.i.d. N(0,1) matrices for edge-case tests.

Host variants return numpy arrays; ``*_device`` variants build the same
distribution on a CUDA device with torch (used for the full-size workloads,
which are too large to build on the host).
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian",
    "haar",
    "haar_spectrum",
    "lowrank_noise",
    "lowrank_noise_device",
    "rbf_points",
    "rbf_bandwidth",
    "rbf_kernel",
    "rbf_kernel_device",
    "psd_lowrank",
    "exact_rank",
    "request_stream",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def gaussian(n: int, m: int, seed: int, dtype=np.float64) -> np.ndarray:
    """i.i.d. standard normal n x m matrix (row-major)."""
    return _rng(seed).standard_normal((n, m)).astype(dtype)


def haar(n: int, k: int, rng: np.random.Generator) -> np.ndarray:
    """n x k matrix with Haar-distributed orthonormal columns.

    QR of a Gaussian matrix with the signs of diag(R) folded into Q
    (Mezzadri 2007), so the distribution is exactly Haar.
    """
    g = rng.standard_normal((n, k))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d


def haar_spectrum(n: int = 4096, m: int = 256, seed: int = 1235,
                  decay: float = 10.0) -> tuple[np.ndarray, np.ndarray]:
    """A = U diag(sigma) V^T, sigma_i = exp(-i/decay), i = 1..min(n,m).

    Returns (A, sigma). FP64.
    """
    rng = _rng(seed)
    k = min(n, m)
    u = haar(n, k, rng)
    v = haar(m, k, rng)
    sigma = np.exp(-np.arange(1, k + 1) / decay)
    a = (u * sigma) @ v.T
    return np.ascontiguousarray(a), sigma


def exact_rank(n: int, m: int, rank: int, seed: int) -> np.ndarray:
    """A matrix of exact rank ``rank`` with singular values 1..1/rank (FP64)."""
    rng = _rng(seed)
    u = haar(n, rank, rng)
    v = haar(m, rank, rng)
    sigma = 1.0 / np.arange(1, rank + 1)
    return np.ascontiguousarray((u * sigma) @ v.T)


def psd_lowrank(n: int, rank: int, seed: int) -> np.ndarray:
    """Symmetric PSD matrix of exact rank ``rank`` (FP64)."""
    rng = _rng(seed)
    u = haar(n, rank, rng)
    lam = 1.0 / np.arange(1, rank + 1)
    a = (u * lam) @ u.T
    return np.ascontiguousarray(0.5 * (a + a.T))


def lowrank_noise(n: int, m: int, rank: int = 1000, noise: float = 1e-4,
                  seed: int = 1236, dtype=np.float64) -> np.ndarray:
    """Host version of G1 diag(i^-2) G2^T + noise * N (orthonormalised G1, G2)."""
    rng = _rng(seed)
    rank = min(rank, n, m)
    g1 = haar(n, rank, rng)
    g2 = haar(m, rank, rng)
    sigma = np.arange(1, rank + 1, dtype=np.float64) ** -2.0
    a = (g1 * sigma) @ g2.T + noise * rng.standard_normal((n, m))
    return np.ascontiguousarray(a.astype(dtype))


def _orthonormalize_device(g, torch):
    """Orthonormal basis of the columns of the tall device matrix g: Gram on
    the device, eigen-decomposition of the small Gram on the host (numpy),
    then g V diag(lambda^-1/2) twice (Gaussian g is well conditioned)."""
    for _ in range(2):
        gram = (g.T @ g).double().cpu().numpy()
        lam, v = np.linalg.eigh(0.5 * (gram + gram.T))
        w = torch.from_numpy(v / np.sqrt(lam)).to(device=g.device, dtype=g.dtype)
        g = g @ w
    return g


def lowrank_noise_device(n: int, m: int, rank: int = 1000, noise: float = 1e-4,
                         seed: int = 1236, dtype=None, device="cuda"):
    """Device version of :func:`lowrank_noise` (torch; same distribution).

    G1 and G2 are Gaussian factors with orthonormalised columns; A is built in
    row panels so that the peak extra memory stays near one copy of A.
    """
    import torch

    dtype = dtype or torch.float32
    work = torch.float64 if dtype == torch.float64 else torch.float32
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    rank = min(rank, n, m)
    g1 = _orthonormalize_device(torch.randn(n, rank, generator=gen, device=device, dtype=work), torch)
    g2 = _orthonormalize_device(torch.randn(m, rank, generator=gen, device=device, dtype=work), torch)
    sigma = torch.arange(1, rank + 1, device=device, dtype=work) ** -2.0
    g2s = (g2 * sigma).T.contiguous()
    a = torch.empty(n, m, device=device, dtype=dtype)
    step = 1 << 16
    for r0 in range(0, n, step):
        r1_ = min(n, r0 + step)
        blk = g1[r0:r1_] @ g2s
        blk += noise * torch.randn(r1_ - r0, m, generator=gen, device=device, dtype=work)
        a[r0:r1_] = blk.to(dtype)
    del g1, g2, g2s
    return a


def psd_lowrank_device(n: int, rank: int = 1000, seed: int = 1241, dtype=None, device="cuda"):
    """Symmetric PSD n x n matrix G diag(i^-2) G^T on the device (G Gaussian
    with orthonormalised columns): the config-2 spectrum for Nystrom requests."""
    import torch

    dtype = dtype or torch.float32
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    rank = min(rank, n)
    g = _orthonormalize_device(torch.randn(n, rank, generator=gen, device=device, dtype=torch.float32), torch)
    sigma = torch.arange(1, rank + 1, device=device, dtype=torch.float32) ** -2.0
    a = torch.empty(n, n, device=device, dtype=dtype)
    gs = (g * sigma).T.contiguous()
    step = 1 << 14
    for r0 in range(0, n, step):
        r1_ = min(n, r0 + step)
        a[r0:r1_] = (g[r0:r1_] @ gs).to(dtype)
    return a


def rbf_points(n: int, d: int = 784, seed: int = 1238, dtype=np.float32) -> np.ndarray:
    """x_i ~ U[0,1]^d, i < n (row-major n x d)."""
    return _rng(seed).random((n, d)).astype(dtype)


def rbf_bandwidth(x: np.ndarray, sub: int = 4096, seed: int = 1239) -> float:
    """Lower median of the pairwise distances |xi - xj| (i < j) over a seeded
    subsample of ``sub`` points (all points when n <= sub)."""
    n = x.shape[0]
    rng = _rng(seed)
    idx = np.sort(rng.choice(n, size=min(sub, n), replace=False))
    xs = x[idx].astype(np.float64)
    sq = np.sum(xs * xs, axis=1)
    d2 = sq[:, None] + sq[None, :] - 2.0 * (xs @ xs.T)
    iu = np.triu_indices(xs.shape[0], k=1)
    dist = np.sqrt(np.maximum(d2[iu], 0.0))
    dist.sort()
    return float(dist[(dist.size - 1) // 2])


def rbf_kernel(x: np.ndarray, h: float, dtype=np.float64) -> np.ndarray:
    """A_ij = exp(-|xi - xj|^2 / (2 h^2)); exactly symmetric, unit diagonal."""
    xs = x.astype(np.float64)
    sq = np.sum(xs * xs, axis=1)
    d2 = np.maximum(sq[:, None] + sq[None, :] - 2.0 * (xs @ xs.T), 0.0)
    d2 = np.triu(d2, 1)
    d2 = d2 + d2.T
    return np.exp(-d2 / (2.0 * h * h)).astype(dtype)


def rbf_kernel_device(x, h: float, dtype=None, tile: int = 8192):
    """Device RBF kernel matrix from points ``x`` (torch, n x d on a GPU).

    Tiles above the diagonal are computed once and mirrored, so A is exactly
    symmetric; the diagonal is exactly one.
    """
    import torch

    dtype = dtype or torch.float32
    n = x.shape[0]
    xw = x.to(torch.float32)
    sq = (xw * xw).sum(dim=1)
    a = torch.empty(n, n, device=x.device, dtype=dtype)
    inv = -1.0 / (2.0 * h * h)
    for i0 in range(0, n, tile):
        i1 = min(n, i0 + tile)
        for j0 in range(i0, n, tile):
            j1 = min(n, j0 + tile)
            d2 = sq[i0:i1, None] + sq[None, j0:j1] - 2.0 * (xw[i0:i1] @ xw[j0:j1].T)
            blk = torch.exp(d2.clamp_(min=0.0) * inv)
            if i0 == j0:
                blk = torch.triu(blk, 1)
                blk = blk + blk.T
                blk.fill_diagonal_(1.0)
            a[i0:i1, j0:j1] = blk.to(dtype)
            if j0 != i0:
                a[j0:j1, i0:i1] = blk.T.to(dtype)
    return a


def request_stream(count: int, seed: int = 1240, rate_hz: float = 100.0, nystrom_max_log2n: int = 15):
    """Poisson stream of mixed requests (sketch / rSVD / Nystrom).

    n = 2^U{14..20}, m log-uniform on [64, 4096], p in {1,2,4,8,16},
    l log-uniform on [64, 1024], target rank k = max(1, l // 4).  An rSVD
    needs l <= min(n, m), so l is capped at m there.  A Nystrom request works
    on an n x n PSD matrix, so its n is drawn from 2^U{14..nystrom_max_log2n}
    (an n x n FP32 matrix at n = 2^20 would need 4 TB).  Returns a list of
    dicts with arrival time ``t`` in seconds.
    """
    rng = _rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=count))
    out = []
    for i in range(count):
        kind = ("sketch", "rsvd", "nystrom")[int(rng.integers(0, 3))]
        n = 1 << int(rng.integers(14, 21))
        m = int(round(float(np.exp(rng.uniform(np.log(64), np.log(4096))))))
        p = int((1, 2, 4, 8, 16)[int(rng.integers(0, 5))])
        l = int(round(float(np.exp(rng.uniform(np.log(64), np.log(1024))))))
        s = int(rng.integers(0, 1 << 62))
        if kind == "rsvd":
            l = min(l, m)
        if kind == "nystrom":
            n = 1 << int(rng.integers(14, nystrom_max_log2n + 1))
            m = n
        out.append({"t": float(t[i]), "kind": kind, "n": n, "m": m, "p": p, "l": l, "k": max(1, l // 4),
                    "seed": s})
    return out
