"""Primal-dual warm starts (Section 6.2's state: z, y, the sketch, p and tau).

A MaxCut SDP is solved to relative gap and infeasibility 1e-3; a neighbouring
instance (the same graph with 1% of its edges moved) is then solved cold and
from the first solve's final iterate with the iteration counter at a quarter
of its final value.  On the FP64 oracle this took 2,396 iterations against
3,135 cold (n = 1,000, 5,000 edges; 2,351 against 3,107 with 5% moved), while
restarting from the dual alone did not help.  Here the GPU paths are held to
the same effect: the warm solve converges and needs clearly fewer iterations.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

N, M, TOL, T_MAX = 1000, 5000, 1e-3, 8000


@pytest.fixture(scope="module")
def S():
    from paper_1912_02949_gb300 import build, scgal
    build.build()
    scgal.load()
    return scgal


def _graphs():
    g = W.er_graph(N, M, seed=11, weights="unit")
    rng = np.random.default_rng(3)
    i2, j2 = g.i.copy(), g.j.copy()
    keys = set(zip(np.minimum(i2, j2).tolist(), np.maximum(i2, j2).tolist()))
    for e in rng.choice(g.i.size, g.i.size // 100, replace=False):
        while True:
            u, v = (int(a) for a in rng.integers(0, N, 2))
            if u != v and (min(u, v), max(u, v)) not in keys:
                keys.add((min(u, v), max(u, v)))
                i2[e], j2[e] = u, v
                break
    csr = [g.csr()[:2], W.csr_from_edges(N, i2, j2, g.w)[:2]]
    return csr


def _params(S, **kw):
    return S.scgal_params_default(R=10, T_max=T_MAX, tol=TOL, precision=32, seed=0, **kw)


def test_standalone_warm_start_from_state(S):
    (rp, col), (rp2, col2) = _graphs()
    a = S.scgal_create_maxcut(rp, col, None, N, col.size, 0.0, _params(S))
    rc, last = S.scgal_solve(a, T_MAX)
    assert rc == S.SCGAL_OK
    st = S.scgal_get_state(a)
    cold = S.scgal_create_maxcut(rp2, col2, None, N, col2.size, 0.0, _params(S))
    rc_c, last_c = S.scgal_solve(cold, T_MAX)
    assert rc_c == S.SCGAL_OK
    warm = S.scgal_create_maxcut(rp2, col2, None, N, col2.size, 0.0, _params(S))
    t0 = max(1, st["t"] // 4)
    S.scgal_set_state(warm, z=st["z"], y=st["y"], S=st["S"], p=st["p"], tau=st["tau"], t=t0)
    rc_w, last_w = S.scgal_solve(warm, T_MAX)
    assert rc_w == S.SCGAL_OK
    it_cold, it_warm = last_c["t"], last_w["t"] - t0 + 1
    assert it_warm < 0.9 * it_cold, (it_warm, it_cold)
    assert last_w["relgap"] <= TOL and last_w["infeas"] <= TOL


def test_served_warm_start(S):
    (rp, col), (rp2, col2) = _graphs()
    srv = S.scgal_server_create(1 << 32, 16)
    ta = S.scgal_submit(srv, rp, col, None, N, col.size, _params(S, keep_state=1))
    ra = S.scgal_poll(srv, ta, -1)
    assert ra["status"] == S.SCGAL_OK and ra["first_t"] == 1
    tw = S.scgal_submit(srv, rp2, col2, None, N, col2.size, _params(S, warm_from=ta))
    tc = S.scgal_submit(srv, rp2, col2, None, N, col2.size, _params(S))
    rw, rcold = S.scgal_poll(srv, tw, -1), S.scgal_poll(srv, tc, -1)
    assert rw["status"] == S.SCGAL_OK and rcold["status"] == S.SCGAL_OK
    assert rw["first_t"] == max(1, (ra["iterations"] + 1) // 4)
    assert rcold["first_t"] == 1
    assert rw["iterations"] < 0.9 * rcold["iterations"], (rw["iterations"], rcold["iterations"])
    # a source that was not kept, or of another size, is a cold start
    tn = S.scgal_submit(srv, rp2, col2, None, N, col2.size, _params(S, warm_from=tc))
    assert S.scgal_poll(srv, tn, -1)["first_t"] == 1
    S.scgal_server_destroy(srv)
