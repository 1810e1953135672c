"""Serving loop (prrp_server_*) on GB300: continuous batching of solve requests.

* every served solution reaches FP64-level normwise backward error (eta <= 1e-15, checked
  on the host in FP64);
* a request's result is bit-identical when served alone and inside a busy mix;
* admission respects the HBM budget (peak working set <= budget; a request that can never
  fit is refused with PRRP_ERR_BUSY), and lanes overlap on the device;
* a singular request fails alone, the others are unaffected; waits can time out.
"""
import numpy as np
import pytest

import prrp_inputs as pi
from oracle import metrics as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prrp():
    import paper_1208_2451_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(prrp):
    c = prrp.prrp_create(0)
    yield c
    c.close()


def _req(n, nrhs, seed):
    return pi.randn(n, seed), pi.rhs(n, nrhs, seed), np.zeros((n, nrhs))


def _serve(prrp, ctx, reqs, budget=64 << 30, lanes=4):
    srv = prrp.prrp_server_create(ctx, budget, lanes=lanes)
    try:
        tickets = [srv.submit(A, B, X) for A, B, X in reqs]
        res = [srv.wait(t) for t in tickets]
        return res, srv.stats()
    finally:
        srv.close()


def test_serve_mixed_requests(prrp, ctx):
    t, ns, nr = pi.serve_requests(40, 1000.0, 64, 2048, 16, 5)
    reqs = [_req(int(n), int(k), 100 + i) for i, (n, k) in enumerate(zip(ns, nr))]
    res, st = _serve(prrp, ctx, reqs)
    assert st["completed"] == 40 and st["rejected"] == 0
    for (A, B, X), r in zip(reqs, res):
        assert r["status"] == 0, r
        for c in range(B.shape[1]):
            assert M.eta(A, X[:, c], B[:, c]) <= 1e-15
    assert st["p99_us"] >= st["p50_us"] > 0


def test_serve_same_alone_and_in_mix(prrp, ctx):
    small = _req(300, 3, 7)
    big = _req(1500, 2, 8)
    alone_s = _serve(prrp, ctx, [small])[0]
    xs_alone = small[2].copy()
    alone_b = _serve(prrp, ctx, [big])[0]
    xb_alone = big[2].copy()
    assert alone_s[0]["status"] == 0 and alone_b[0]["status"] == 0
    small[2][:] = 0.0
    big[2][:] = 0.0
    _, ns, nr = pi.serve_requests(30, 1000.0, 64, 1400, 8, 11)
    mix = [_req(int(n), int(k), 300 + i) for i, (n, k) in enumerate(zip(ns, nr))]
    mix.insert(5, small)
    mix.insert(17, big)
    res, st = _serve(prrp, ctx, mix)
    assert all(r["status"] == 0 for r in res), [(A.shape[0], r) for (A, _, _), r in zip(mix, res)
                                                if r["status"] != 0]
    assert np.array_equal(small[2], xs_alone)
    assert np.array_equal(big[2], xb_alone)
    assert st["peak_busy_lanes"] >= 2, st        # lanes overlapped on the device


def test_serve_admission_budget(prrp, ctx):
    reqs = [_req(n, 1, 40 + n) for n in (1200, 1300, 1100, 200, 150)]
    budget = 16 * 1300 * 1300 + 40 * 1300 + 1024 * 1300 + 4096 + 64 * 2**20
    res, st = _serve(prrp, ctx, reqs, budget=budget, lanes=3)
    assert all(r["status"] == 0 for r in res)
    assert st["peak_bytes_in_use"] <= budget
    srv = prrp.prrp_server_create(ctx, 1 << 20, lanes=1)
    try:
        A, B, X = _req(2000, 1, 1)
        with pytest.raises(prrp.PrrpError) as e:
            srv.submit(A, B, X)
        assert e.value.name == "PRRP_ERR_BUSY"
    finally:
        srv.close()


def test_serve_failure_and_timeout(prrp, ctx):
    bad = _req(128, 1, 3)
    bad[0][:, 32:48] = 0.0
    good = _req(128, 1, 4)
    big = _req(3000, 1, 5)
    srv = prrp.prrp_server_create(ctx, 64 << 30, lanes=2)
    try:
        tb = srv.submit(*big)
        with pytest.raises(prrp.PrrpError) as e:
            srv.wait(tb, timeout_us=0)
        assert e.value.name == "PRRP_ERR_TIMEOUT"
        t1, t2 = srv.submit(*bad), srv.submit(*good)
        r1, r2, rb = srv.wait(t1), srv.wait(t2), srv.wait(tb)
        assert r1["status"] == prrp.binding.PRRP_ERR_SINGULAR
        assert r2["status"] == 0 and rb["status"] == 0
        assert M.eta(big[0], big[2][:, 0], big[1][:, 0]) <= 1e-15
    finally:
        srv.close()
