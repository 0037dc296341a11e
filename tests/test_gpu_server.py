"""Serving loop: continuous batching, admission by device footprint, and each
result equal alone and in the mix."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_1912_02949_gb300 import build, scgal
    build.build()
    scgal.load()
    return scgal


def _requests(k, seed=0):
    reqs = W.serving_requests(k, rate=1000.0, seed=seed, n_lo=100, n_hi=3000)
    out = []
    for r in reqs:
        g = W.er_graph(r["n"], r["m"], seed=r["seed"], weights="unit")
        rp, col, _ = g.csr()
        out.append((r, g, rp, col))
    return out


def _params(S, r):
    return S.scgal_params_default(R=10, T_max=400, tol=1e-2, precision=32, seed=r["seed"], instance=r["id"])


def test_alone_equals_mixed(S):
    reqs = _requests(24)
    srv = S.scgal_server_create(1 << 34, 8)
    tickets = []
    for r, g, rp, col in reqs:
        tickets.append(S.scgal_submit(srv, rp, col, None, g.n, col.size, _params(S, r)))
        time.sleep(0.002)   # arrivals spread while earlier solves are running
    mixed = [S.scgal_poll(srv, t, -1) for t in tickets]
    st = S.scgal_server_get_stats(srv)
    S.scgal_server_destroy(srv)
    assert st["completed"] == len(reqs) and st["rejected"] == 0
    for (r, g, rp, col), res in zip(reqs, mixed):
        assert res["status"] in (S.SCGAL_OK, S.SCGAL_ENOTDONE)
        h = S.scgal_create_maxcut(rp, col, None, g.n, col.size, 0.0, _params(S, r))
        rc, last = S.scgal_solve(h, 400)
        _, lam, _, cut = S.scgal_reconstruct(h)
        h.close()
        assert res["status"] == rc
        assert res["iterations"] == (last["t"] - 1 if last["converged"] else last["t"])
        assert res["relgap"] == last["relgap"] and res["infeas"] == last["infeas"]
        assert res["objective"] == last["p"] and res["best_cut"] == cut
        assert res["lambda_max"] == lam[0]
        assert res["latency_ms"] >= res["queue_ms"] >= 0.0


def test_admission_by_budget_and_rejection(S):
    reqs = _requests(6, seed=1)
    budget = 8 << 20      # a few of these solves at once, not all six
    srv = S.scgal_server_create(budget, 8)
    tickets = [S.scgal_submit(srv, rp, col, None, g.n, col.size, _params(S, r)) for r, g, rp, col in reqs]
    res = [S.scgal_poll(srv, t, -1) for t in tickets]
    st = S.scgal_server_get_stats(srv)
    assert 0 < st["device_bytes_peak"] <= budget
    assert all(x["status"] in (S.SCGAL_OK, S.SCGAL_ENOTDONE) for x in res)
    # a request that can never fit is rejected, not queued forever
    big = W.er_graph(200000, 600000, seed=3)
    rp, col, _ = big.csr()
    t = S.scgal_submit(srv, rp, col, None, big.n, col.size, S.scgal_params_default(T_max=100))
    out = S.scgal_poll(srv, t, 60000)
    assert out["status"] == S.SCGAL_ENOMEM
    S.scgal_server_destroy(srv)


def test_poll_timeout_and_unknown_ticket(S):
    srv = S.scgal_server_create(1 << 32, 2)
    assert S.scgal_poll(srv, 12345, 0) is None
    g = W.er_graph(2000, 8000, seed=4)
    rp, col, _ = g.csr()
    t = S.scgal_submit(srv, rp, col, None, g.n, col.size, S.scgal_params_default(T_max=300, tol=1e-9))
    assert S.scgal_poll(srv, t, 0) is None            # not finished yet
    assert S.scgal_poll(srv, t, -1) is not None
    S.scgal_server_destroy(srv)
