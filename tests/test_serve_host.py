"""Host-side parts of the serving loop (no GPU): the scratch pool's first-fit
allocator against a byte-map model, and the request-stream generator's
distributions."""

import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def lib():
    import paper_2210_11295_gb300 as b
    return b


@pytest.mark.parametrize("seed", [1, 2, 3, 12345])
def test_pool_allocator_matches_model(lib, seed):
    assert lib.bsrht_selftest_pool_allocator(seed, 20000) == 0


def test_request_stream_distribution():
    rate = 100.0
    reqs = synth.request_stream(10000, seed=1240, rate_hz=rate)
    t = np.array([r["t"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    # Exponential gaps: mean 1/rate, coefficient of variation 1.
    assert abs(gaps.mean() * rate - 1.0) < 0.05
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05
    kinds = [r["kind"] for r in reqs]
    for k in ("sketch", "rsvd", "nystrom"):
        assert abs(kinds.count(k) / len(reqs) - 1 / 3) < 0.03
    for r in reqs:
        assert r["p"] in (1, 2, 4, 8, 16)
        assert r["n"] & (r["n"] - 1) == 0
        if r["kind"] == "nystrom":
            assert 1 << 14 <= r["n"] <= 1 << 15 and r["m"] == r["n"]
        else:
            assert 1 << 14 <= r["n"] <= 1 << 20 and 64 <= r["m"] <= 4096
        assert 64 <= r["l"] <= 1024 and 1 <= r["k"] <= r["l"]
        if r["kind"] == "rsvd":
            assert r["l"] <= r["m"]
    # Log-uniform m: the median of log m sits at the middle of [log 64, log 4096].
    lm = np.log([r["m"] for r in reqs if r["kind"] != "nystrom"])
    assert abs(np.median(lm) - 0.5 * (np.log(64) + np.log(4096))) < 0.1
