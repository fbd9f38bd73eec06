"""The Gaussian-embedding comparator (BSRHT_VARIANT_GAUSSIAN) on the GPU
against the CPU oracle (oracle.gaussian), through the C ABI.

Parity bar: the FP32 one, relative Frobenius 1e-5 (the entries of Omega_G
come from the same counter-based generator on both sides; the GPU evaluates
Box-Muller in FP32 and the product at FP32 accuracy).  Also: repeated calls
give identical bits, rSVD with the Gaussian sketch matches the oracle's
Algorithm 1 with the same Omega_G, the paper's observation that the Gaussian
and block SRHT sketches give the same approximation quality (Sec. 4), sampled
entries at the full benchmark size, and the unsupported combinations."""

import numpy as np
import pytest
import torch

from oracle import gaussian as og
from oracle import lowrank as orl
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_11295_gb300 as b
    return b


def _rel(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


@pytest.mark.parametrize("n,m,l,seed", [
    (4096, 64, 128, 0),
    (5003, 33, 100, 1),    # n and m not multiples of 4 (padded Omega rows, ragged tiles)
    (8, 8, 8, 2),          # smallest n of the tensor-core product
    (20000, 256, 512, 3),  # several M and N tiles, split K
    (3000, 5, 700, 4),     # l > 512, narrow A
])
def test_gaussian_sketch_matches_oracle(lib, n, m, l, seed):
    a = synth.gaussian(n, m, seed=100 + seed).astype(np.float32)
    got = lib.bsrht_sketch(torch.from_numpy(a).cuda(), 1, l, seed, variant=lib.VARIANT_GAUSSIAN)
    torch.cuda.synchronize()
    ref = og.gaussian_sketch(a.astype(np.float64), l, seed)
    assert got.shape == (l, m)
    assert _rel(got.cpu().numpy(), ref) <= 1e-5


def test_gaussian_sketch_row_stride_and_determinism(lib):
    n, m, l = 6000, 40, 64
    a = synth.gaussian(n, m, seed=7).astype(np.float32)
    big = torch.zeros(n, 48, dtype=torch.float32)
    big[:, :m] = torch.from_numpy(a)
    dev = big.cuda()[:, :m]
    b1 = lib.bsrht_sketch(dev, 4, l, 9, variant=lib.VARIANT_GAUSSIAN).clone()
    b2 = lib.bsrht_sketch(dev, 4, l, 9, variant=lib.VARIANT_GAUSSIAN).clone()
    torch.cuda.synchronize()
    assert torch.equal(b1, b2)
    assert _rel(b1.cpu().numpy(), og.gaussian_sketch(a.astype(np.float64), l, 9)) <= 1e-5


def test_rsvd_with_gaussian_sketch_matches_oracle(lib):
    a32 = synth.lowrank_noise(1 << 15, 384, rank=200, seed=12, dtype=np.float32)
    k, l = 30, 96
    u, s, v = lib.bsrht_rsvd(torch.from_numpy(a32).cuda(), k, l, 4, 3, variant=lib.VARIANT_GAUSSIAN)
    torch.cuda.synchronize()
    u, s, v = u.cpu().numpy(), s.cpu().numpy(), v.cpu().numpy()
    a64 = a32.astype(np.float64)
    ur, sr, vr = orl.rsvd(a64, k, l, 4, 3, sketch="gaussian")
    assert np.max(np.abs(s - sr)) <= 2e-5 * sr[0]
    err = np.linalg.norm(a64 - (u * s) @ v.T)
    err_ref = np.linalg.norm(a64 - (ur * sr) @ vr.T)
    assert abs(err - err_ref) <= 1e-4 * err_ref
    assert np.linalg.norm(u.T @ u - np.eye(k)) <= 1e-5
    assert np.linalg.norm(v.T @ v - np.eye(k)) <= 1e-5


def test_gaussian_and_block_srht_give_the_same_quality(lib):
    """Sec. 4: the block SRHT and Gaussian sketches give practically identical
    rSVD errors; here within 3 % of each other and of the Eckart-Young
    optimum's scale, on a spectrum with a clear decay (Haar factors)."""
    n, m, k, l = 1 << 15, 256, 20, 60
    a, sig = synth.haar_spectrum(n, m, seed=13)
    opt = np.sqrt(np.sum(np.asarray(sig, dtype=np.float64)[k:] ** 2))
    dev = torch.from_numpy(a.astype(np.float32)).cuda()
    a64 = a.astype(np.float32).astype(np.float64)
    errs = {}
    for name, variant in (("bsrht", lib.VARIANT_AUTO), ("gauss", lib.VARIANT_GAUSSIAN)):
        e = []
        for seed in range(3):
            u, s, v = lib.bsrht_rsvd(dev, k, l, 8, seed, variant=variant)
            torch.cuda.synchronize()
            e.append(np.linalg.norm(a64 - (u.cpu().numpy() * s.cpu().numpy()) @ v.cpu().numpy().T))
        errs[name] = float(np.mean(e))
    assert errs["bsrht"] >= opt * (1 - 1e-6) and errs["gauss"] >= opt * (1 - 1e-6)
    assert abs(errs["bsrht"] / errs["gauss"] - 1.0) <= 0.03


def test_full_size_sampled_entries(lib):
    """n = 2^20, m = 4096, l = 512 (the benchmark's FP32 workload): sampled
    entries B[j, c] = Omega_G[j, :] A[:, c], the oracle forming each sampled
    row of Omega_G from the generator."""
    n, m, l, seed = 1 << 20, 4096, 512, 5
    a = synth.lowrank_noise_device(n, m, seed=1236, dtype=torch.float32)
    b = lib.bsrht_sketch(a, 4, l, seed, variant=lib.VARIANT_GAUSSIAN)
    torch.cuda.synchronize()
    cols = [0, 1, 1000, 4095]
    acols = a[:, cols].double().cpu().numpy()
    bs = b[:, cols].double().cpu().numpy()
    del a, b
    for j in (0, 1, 255, 511):
        om_j = _omega_row(j, n, l, seed)
        ref = om_j @ acols
        scale = np.linalg.norm(om_j) * np.linalg.norm(acols, axis=0)
        assert np.all(np.abs(bs[j] - ref) <= 1e-5 * scale), (j, bs[j], ref)


def _omega_row(j, n, l, seed):
    """Row j of Omega_G from the oracle's generator (counter (k >> 1, j, 3, 0))."""
    npair = (n + 1) // 2
    q = np.arange(npair, dtype=np.uint64)
    w0, w1, w2, w3 = og.philox4x64_10_vec(q, np.full_like(q, j), np.full_like(q, og.STREAM_G), np.zeros_like(q),
                                           seed, 0)
    row = np.empty(2 * npair)
    row[0::2] = og.box_muller(og.uniform_from_word(w0), og.uniform_from_word(w1))
    row[1::2] = og.box_muller(og.uniform_from_word(w2), og.uniform_from_word(w3))
    return row[:n] / np.sqrt(l)


def test_gaussian_unsupported_combinations(lib):
    cases = [
        lambda: lib.bsrht_sketch(torch.zeros(64, 8, device="cuda", dtype=torch.float64), 1, 8, 0,
                                 variant=lib.VARIANT_GAUSSIAN),
        lambda: lib.bsrht_sketch(torch.zeros(64, 8, device="cuda", dtype=torch.bfloat16), 1, 8, 0,
                                 variant=lib.VARIANT_GAUSSIAN),
        lambda: lib.bsrht_sketch(torch.zeros(7, 8, device="cuda", dtype=torch.float32), 1, 4, 0,
                                 variant=lib.VARIANT_GAUSSIAN),
        lambda: lib.bsrht_nystrom(torch.eye(64, device="cuda", dtype=torch.float32), 4, 8, 1, 0,
                                  variant=lib.VARIANT_GAUSSIAN),
    ]
    for f in cases:
        with pytest.raises(lib.BsrhtError) as e:
            f()
        assert e.value.status == -95
