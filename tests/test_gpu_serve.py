"""Serving loop on the GPU (bsrht_server_*): continuous batching, grouped
sketch launches, CUDA-graph replay, admission by HBM footprint, bounded
waits and the sketch autotuner.

The central check: every request gives the same result in a mix of
concurrent requests as alone (one direct library call at a time), within the
parity tolerances (relative Frobenius 1e-12 for FP64 arithmetic, 1e-5 for
FP32).  Grouped sketches are also compared with the CPU oracle."""

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
    got = got.double().cpu().numpy() if isinstance(got, torch.Tensor) else np.asarray(got, np.float64)
    ref = ref.double().cpu().numpy() if isinstance(ref, torch.Tensor) else np.asarray(ref, np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


def _sketch_cases():
    """Small sketches (grouped: too few tiles to fill the GPU) and larger ones
    (single launches), over dtypes, ragged m and every p of the serving mix."""
    cases = []
    rng = np.random.default_rng(5)
    for i in range(18):
        n = 1 << int(rng.integers(14, 16))
        m = int((64, 100, 96, 160)[i % 4])
        p = int((1, 2, 4, 8, 16)[i % 5])
        l = int((64, 100, 200)[i % 3])
        dt = (torch.float32, torch.float64, torch.bfloat16)[i % 3]
        cases.append((n, m, p, l, dt, 100 + i))
    cases += [(1 << 18, 512, 4, 256, torch.float32, 7), (1 << 17, 300, 8, 128, torch.float64, 8),
              (1 << 18, 256, 1, 512, torch.bfloat16, 9)]
    return cases


def _make(n, m, dt, seed):
    return torch.from_numpy(synth.gaussian(n, m, seed=seed)).to(dt).cuda()


def test_mix_equals_alone(lib):
    sk = [(c, _make(c[0], c[1], c[4], c[5])) for c in _sketch_cases()]
    a_r = torch.from_numpy(synth.lowrank_noise(1 << 15, 256, rank=128, seed=21)).cuda()
    a_r32 = a_r.float()
    a_n = torch.from_numpy(synth.psd_lowrank(3000, 40, seed=22)).cuda()
    torch.cuda.synchronize()  # the server's streams do not wait for torch's
    # Alone: one direct call at a time.
    alone_sk = []
    for (n, m, p, l, dt, seed), a in sk:
        alone_sk.append(lib.bsrht_sketch(a, p, l, seed).clone())
    torch.cuda.synchronize()
    alone_r = [lib.bsrht_rsvd(a, 20, 64, 4, 3) for a in (a_r, a_r32)]
    alone_n = lib.bsrht_nystrom(a_n, 30, 60, 4, 2)
    torch.cuda.synchronize()
    alone_r = [tuple(x.clone() for x in t) for t in alone_r]
    alone_n = tuple(x.clone() for x in alone_n)

    # Two executors: the RSVD / Nystrom requests, submitted first, keep them
    # busy while the sketches queue up, so the sketches must be packed into
    # grouped launches when an executor frees up.
    with lib.Server(hbm_budget=2 << 30, executors=2, max_group=16) as srv:
        tickets, outs = [], []
        r_outs = []
        for a in (a_r, a_r32):
            o = (torch.empty(a.shape[0], 20, device="cuda", dtype=torch.float64),
                 torch.empty(20, device="cuda", dtype=torch.float64),
                 torch.empty(a.shape[1], 20, device="cuda", dtype=torch.float64))
            r_outs.append(o)
        n_out = (torch.empty(3000, 30, device="cuda", dtype=torch.float64),
                 torch.empty(30, device="cuda", dtype=torch.float64))
        sk_outs = [torch.empty(l, m, device="cuda", dtype=lib.sketch_out_dtype(dt)) for (n, m, p, l, dt, seed), a in sk]
        r_tickets = [srv.submit_rsvd(a, 20, 64, 4, 3, o) for a, o in zip((a_r, a_r32), r_outs)]
        n_ticket = srv.submit_nystrom(a_n, 30, 60, 4, 2, n_out)
        for ((n, m, p, l, dt, seed), a), out in zip(sk, sk_outs):
            tickets.append(srv.submit_sketch(a, p, l, seed, out))
            outs.append(out)
        tickets += r_tickets + [n_ticket]
        for t in tickets:
            assert srv.wait(t, 600.0) == 0
        st = srv.stats()
    assert st["completed"] == st["submitted"] == len(tickets) and st["failed"] == 0
    assert st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    assert st["grouped_requests"] > st["grouped_launches"] > 0  # some launch packed >= 2 sketches
    assert st["graph_launches"] > 0
    for ((n, m, p, l, dt, seed), a), out, ref in zip(sk, outs, alone_sk):
        assert _rel(out, ref) <= TOL[dt], (n, m, p, l, dt)
    for got, ref, dt in zip(r_outs, alone_r, (torch.float64, torch.float32)):
        tol = TOL[dt]
        assert _rel(got[1], ref[1]) <= tol
        assert _rel((got[0] * got[1]) @ got[2].T, (ref[0] * ref[1]) @ ref[2].T) <= 10 * tol
    assert _rel(n_out[1], alone_n[1]) <= 1e-12
    assert _rel((n_out[0] * n_out[1]) @ n_out[0].T, (alone_n[0] * alone_n[1]) @ alone_n[0].T) <= 1e-10


def test_grouped_sketch_matches_oracle(lib):
    """FP64 small sketches that the server packs into grouped launches,
    against the CPU oracle (relative Frobenius 1e-12)."""
    cases = [(1 << 14, 64, 4, 64, 1), (1 << 14, 100, 16, 128, 2), (1 << 14, 33, 3, 100, 3),
             (20000, 64, 5, 90, 4), (1 << 14, 96, 1, 64, 5)]
    data = [synth.gaussian(n, m, seed=seed) for n, m, p, l, seed in cases]
    dev = [torch.from_numpy(a).cuda() for a in data]
    torch.cuda.synchronize()
    with lib.Server(hbm_budget=1 << 30, executors=1, max_group=8, autotune=False) as srv:
        outs, tickets = [], []
        for (n, m, p, l, seed), a in zip(cases, dev):
            out = torch.empty(l, m, device="cuda", dtype=torch.float64)
            tickets.append(srv.submit_sketch(a, p, l, seed, out))
            outs.append(out)
        for t in tickets:
            assert srv.wait(t, 600.0) == 0
        st = srv.stats()
    assert st["grouped_requests"] == len(cases)
    for (n, m, p, l, seed), a, out in zip(cases, data, outs):
        ref = orc.sketch_fast(a, p, l, seed)
        assert _rel(out, ref) <= 1e-12, (n, m, p, l)


def test_admission_by_footprint(lib):
    """A budget that holds one request at a time still completes them all
    (they queue for memory); a request larger than the budget is refused."""
    a = torch.from_numpy(synth.gaussian(1 << 16, 256, seed=31)).float().cuda()
    need = lib.bsrht_rsvd_workspace(1 << 16, 256, 16, 64, 4, torch.float32)
    budget = int(need * 1.5)
    torch.cuda.synchronize()
    with lib.Server(hbm_budget=budget, executors=4) as srv:
        outs, tickets = [], []
        for i in range(6):
            o = (torch.empty(1 << 16, 16, device="cuda", dtype=torch.float64),
                 torch.empty(16, device="cuda", dtype=torch.float64),
                 torch.empty(256, 16, device="cuda", dtype=torch.float64))
            tickets.append(srv.submit_rsvd(a, 16, 64, 4, i, o))
            outs.append(o)
        big = torch.from_numpy(synth.gaussian(1 << 17, 512, seed=32)).float().cuda()
        torch.cuda.synchronize()
        ob = (torch.empty(1 << 17, 16, device="cuda", dtype=torch.float64),
              torch.empty(16, device="cuda", dtype=torch.float64),
              torch.empty(512, 16, device="cuda", dtype=torch.float64))
        with pytest.raises(lib.BsrhtError) as e:
            srv.submit_rsvd(big, 16, 256, 4, 0, ob)
        assert e.value.status == -12
        for t in tickets:
            assert srv.wait(t, 600.0) == 0
        st = srv.stats()
    assert st["completed"] == 6 and st["failed"] == 0
    assert st["pool_high_bytes"] <= budget
    for i, o in enumerate(outs):
        ref = lib.bsrht_rsvd(a, 16, 64, 4, i)
        assert _rel(o[1], ref[1]) <= 1e-5


def test_bounded_wait_times_out(lib):
    """bsrht_wait returns ETIMEDOUT for a request still running and the
    request's status once it has finished."""
    a = torch.from_numpy(synth.gaussian(1 << 18, 1024, seed=41)).float().cuda()
    torch.cuda.synchronize()
    with lib.Server(hbm_budget=4 << 30, executors=1) as srv:
        o = (torch.empty(1 << 18, 32, device="cuda", dtype=torch.float64),
             torch.empty(32, device="cuda", dtype=torch.float64),
             torch.empty(1024, 32, device="cuda", dtype=torch.float64))
        t = srv.submit_rsvd(a, 32, 512, 4, 0, o)
        assert srv.wait(t, 0.0) == -110
        done, st = srv.poll(t)
        assert not done and st == 0
        assert srv.wait(t, 600.0) == 0
        done, st = srv.poll(t)
        assert done and st == 0


def test_autotune_keeps_results(lib):
    a = _make(1 << 18, 512, torch.float32, 51)
    ref = lib.bsrht_sketch(a, 4, 256, 9).clone()
    lib.bsrht_sketch_autotune_reset()
    try:
        choice, ms = lib.bsrht_sketch_autotune(a, 4, 256)
        assert -1 <= choice <= 6 and ms > 0
        got = lib.bsrht_sketch(a, 4, 256, 9)
        assert _rel(got, ref) <= 1e-5
    finally:
        lib.bsrht_sketch_autotune_reset()
