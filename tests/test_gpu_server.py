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


def _result_fields(r):
    # the solve's results; timings and the server's learned work estimate
    # (predicted_iterations, which grows as finished requests teach it) vary
    return {k: v for k, v in r.items() if k not in ("queue_ms", "latency_ms", "predicted_iterations")}


def test_alone_equals_mixed(S):
    """Each request's result is identical whether it is solved alone or among
    others that arrive while it is running (continuous batching)."""
    reqs = _requests(24)
    srv = S.scgal_server_create(1 << 34, 8)
    tickets = []
    for r, g, rp, col in reqs:
        tickets.append(S.scgal_submit(srv, rp, col, None, g.n, col.size, _params(S, r)))
        time.sleep(0.002)   # arrivals spread while earlier solves are running
    mixed = [S.scgal_poll(srv, t, -1) for t in tickets]
    st = S.scgal_server_get_stats(srv)
    assert st["completed"] == len(reqs) and st["rejected"] == 0
    for (r, g, rp, col), res in zip(reqs, mixed):   # now one at a time on the idle server
        alone = S.scgal_poll(srv, S.scgal_submit(srv, rp, col, None, g.n, col.size, _params(S, r)), -1)
        assert res["status"] in (S.SCGAL_OK, S.SCGAL_ENOTDONE)
        assert _result_fields(res) == _result_fields(alone)
        assert res["latency_ms"] >= res["queue_ms"] >= 0.0
    S.scgal_server_destroy(srv)


def test_served_solve_matches_oracle():
    """A request solved by the server's batched engine against the FP64 oracle:
    n = 800 Erdos-Renyi MaxCut, T = 500: objective within 1e-3 relative, the
    rounded cut within the oracle's own spread (see test_gpu_maxcut)."""
    from paper_1912_02949_gb300 import scgal as S
    from oracle.problems import MaxCutProblem
    from oracle.sketchycgal import sketchy_cgal
    S.load()
    g = W.config_graph("er800")
    rp, col, _ = g.csr()
    srv = S.scgal_server_create(1 << 32, 2)
    res = S.scgal_poll(srv, S.scgal_submit(srv, rp, col, None, g.n, col.size,
                                           S.scgal_params_default(R=10, T_max=500, precision=32)), -1)
    S.scgal_server_destroy(srv)
    ref = sketchy_cgal(MaxCutProblem(g.n, g.i, g.j, g.w), R=10, T=500, seed=0).history[-1]
    assert res["status"] == S.SCGAL_ENOTDONE and res["iterations"] == 500
    assert abs(res["objective"] - ref["p_orig"]) <= 1e-3 * abs(ref["p_orig"])
    assert 0 < res["best_cut"] <= 19176


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


def test_alone_equals_mixed_with_clustered_instances(S):
    """Instances with n >= 16384 run on a cluster of four blocks (x copied into
    every block's shared memory, sums combined across the cluster in a fixed
    order); their results, and those of small instances sharing the rounds, are
    identical alone and mixed."""
    sizes = [(20000, 8), (300, 6), (40000, 6), (1500, 10), (17000, 12), (800, 8)]
    reqs = []
    for k, (n, deg) in enumerate(sizes):
        g = W.er_graph(n, n * deg // 2, seed=100 + k, weights="unit" if k % 3 else "pm1")
        rp, col, val = g.csr()
        reqs.append((k, g, rp, col, val if g.weight_kind != "unit" else None))

    def prm(k):
        return S.scgal_params_default(R=10, T_max=60, tol=0.0, precision=32, seed=7, instance=k)

    srv = S.scgal_server_create(1 << 34, 8)
    tickets = [S.scgal_submit(srv, rp, col, val, g.n, col.size, prm(k)) for k, g, rp, col, val in reqs]
    mixed = [S.scgal_poll(srv, t, -1) for t in tickets]
    for (k, g, rp, col, val), res in zip(reqs, mixed):
        alone = S.scgal_poll(srv, S.scgal_submit(srv, rp, col, val, g.n, col.size, prm(k)), -1)
        assert res["status"] == S.SCGAL_ENOTDONE and res["iterations"] == 60
        assert _result_fields(res) == _result_fields(alone)
    S.scgal_server_destroy(srv)


def test_clustered_solve_matches_oracle():
    """A clustered instance (n = 20000, unit weights) served against the FP64
    oracle on the same random draws.  After one update (the record of t = 2) the
    trajectories still coincide: objective and infeasibility to 1e-5 relative.
    At T = 150 every FP32 path, the per-handle graph path included, sits about
    0.5% from the FP64 trajectory on this graph (measured: graph path -64786,
    clustered -64677, oracle -65101; the oracle's own spread under 1e-7
    perturbations of its start vectors is 1e-4), so the bar there is 1.5%
    on the objective and 5% on the infeasibility."""
    from paper_1912_02949_gb300 import scgal as S
    from oracle.problems import MaxCutProblem
    from oracle.sketchycgal import sketchy_cgal
    S.load()
    g = W.er_graph(20000, 80000, seed=5, weights="unit")
    rp, col, _ = g.csr()
    srv = S.scgal_server_create(1 << 33, 2)
    res = {}
    for T in (2, 150):
        res[T] = S.scgal_poll(srv, S.scgal_submit(srv, rp, col, None, g.n, col.size,
                                                  S.scgal_params_default(R=10, T_max=T, tol=0.0, precision=32)), -1)
    S.scgal_server_destroy(srv)
    hist = sketchy_cgal(MaxCutProblem(g.n, g.i, g.j, g.w), R=10, T=150, seed=0).history
    for T, rtol_p, rtol_i in ((2, 1e-5, 1e-5), (150, 1.5e-2, 5e-2)):
        ref = hist[T - 1]
        assert res[T]["status"] == S.SCGAL_ENOTDONE and res[T]["iterations"] == T
        assert abs(res[T]["objective"] - ref["p_orig"]) <= rtol_p * abs(ref["p_orig"])
        assert abs(res[T]["infeas"] - ref["infeas"]) <= rtol_i * ref["infeas"]


@pytest.mark.parametrize("n,kind", [(3000, "real"), (20000, "real"), (33000, "pm1"), (20000, "pm1")])
def test_served_weight_kinds_match_oracle(n, kind):
    """Every batched kernel variant against the FP64 oracle after one update
    (the record of t = 2, where FP32 and FP64 trajectories still coincide):
    general weights (value arrays in the sliced layout) in a one-block and a
    clustered instance, +/-1 weights with 32-bit columns (n >= 32767, the sign
    in bit 31) and with 16-bit columns (sign in bit 15)."""
    from paper_1912_02949_gb300 import scgal as S
    from oracle.problems import MaxCutProblem
    from oracle.sketchycgal import sketchy_cgal
    S.load()
    g = W.er_graph(n, 4 * n, seed=11, weights=kind)
    rp, col, val = g.csr()
    srv = S.scgal_server_create(1 << 33, 2)
    res = S.scgal_poll(srv, S.scgal_submit(srv, rp, col, val, g.n, col.size,
                                           S.scgal_params_default(R=10, T_max=2, tol=0.0, precision=32)), -1)
    S.scgal_server_destroy(srv)
    ref = sketchy_cgal(MaxCutProblem(g.n, g.i, g.j, g.w), R=10, T=2, seed=0).history[1]
    assert res["status"] == S.SCGAL_ENOTDONE and res["iterations"] == 2
    assert abs(res["objective"] - ref["p_orig"]) <= 1e-5 * abs(ref["p_orig"])
    assert abs(res["infeas"] - ref["infeas"]) <= 1e-5 * ref["infeas"]


def test_graph_path_requests_share_rounds(S):
    """Requests the batched engine does not take -- FP64, and n above its
    shared-memory limit -- run on their handles' own graphs in the same rounds
    as batched ones; every result is identical alone and mixed."""
    specs = [(1200, "unit", 32), (2500, "pm1", 64), (60000, "unit", 32), (900, "unit", 32), (20000, "unit", 32)]
    reqs = []
    for k, (n, kind, prec) in enumerate(specs):
        g = W.er_graph(n, 4 * n, seed=200 + k, weights=kind)
        rp, col, val = g.csr()
        reqs.append((k, g, rp, col, val if kind != "unit" else None, prec))

    def prm(k, prec):
        return S.scgal_params_default(R=10, T_max=40, tol=0.0, precision=prec, seed=3, instance=k)

    srv = S.scgal_server_create(1 << 34, 8)
    tickets = [S.scgal_submit(srv, rp, col, val, g.n, col.size, prm(k, prec)) for k, g, rp, col, val, prec in reqs]
    mixed = [S.scgal_poll(srv, t, -1) for t in tickets]
    for (k, g, rp, col, val, prec), res in zip(reqs, mixed):
        alone = S.scgal_poll(srv, S.scgal_submit(srv, rp, col, val, g.n, col.size, prm(k, prec)), -1)
        assert res["status"] == S.SCGAL_ENOTDONE and res["iterations"] == 40
        assert _result_fields(res) == _result_fields(alone)
    S.scgal_server_destroy(srv)


@pytest.mark.parametrize("n,m,R", [(2, 1, 2), (50, 0, 10), (300, 900, 1), (300, 900, 5), (300, 900, 16)])
def test_batched_edge_cases_match_oracle(n, m, R):
    """Batched solves at the edges of the engine: the smallest graph, a graph
    without edges (every slice of width 0; C = 0, Eq. 7.1 leaves it unscaled),
    and sketch ranks 1, 5 and 16 (the Ritz step's accumulator widths), against
    the FP64 oracle after one update.  Without edges D_1 = -beta b I is a
    multiple of the identity, every vector is a minimum eigenvector and the one
    Lanczos returns is decided by rounding (the oracle's own infeasibility
    differs between x86 and Arm), so only the exact objective 0 is compared."""
    from paper_1912_02949_gb300 import scgal as S
    from oracle.problems import MaxCutProblem
    from oracle.sketchycgal import sketchy_cgal
    S.load()
    g = W.er_graph(n, m, seed=21, weights="unit")
    rp, col, _ = g.csr()
    srv = S.scgal_server_create(1 << 32, 2)
    res = S.scgal_poll(srv, S.scgal_submit(srv, rp, col, None, g.n, col.size,
                                           S.scgal_params_default(R=R, T_max=2, tol=0.0, precision=32)), -1)
    S.scgal_server_destroy(srv)
    ref = sketchy_cgal(MaxCutProblem(g.n, g.i, g.j, g.w), R=R, T=2, seed=0).history[1]
    assert res["status"] == S.SCGAL_ENOTDONE and res["iterations"] == 2
    assert abs(res["objective"] - ref["p_orig"]) <= 1e-5 * max(abs(ref["p_orig"]), 1.0)
    if m == 0:
        assert res["objective"] == 0.0 and np.isfinite(res["infeas"])
    else:
        assert abs(res["infeas"] - ref["infeas"]) <= 1e-5 * max(ref["infeas"], 1e-3)


def test_batched_solve_converges_early():
    """A loose tolerance: the stopping rule (Eq. E.1) ends the batched solve
    before T_max and the result carries status OK and the iterations run."""
    from paper_1912_02949_gb300 import scgal as S
    S.load()
    g = W.er_graph(2000, 8000, seed=22, weights="unit")
    rp, col, _ = g.csr()
    srv = S.scgal_server_create(1 << 32, 2)
    res = S.scgal_poll(srv, S.scgal_submit(srv, rp, col, None, g.n, col.size,
                                           S.scgal_params_default(R=10, T_max=3000, tol=5e-2, precision=32)), -1)
    S.scgal_server_destroy(srv)
    assert res["status"] == S.SCGAL_OK
    assert 1 <= res["iterations"] < 3000
    assert res["relgap"] <= 5e-2 and res["infeas"] <= 5e-2


def test_served_phase_retrieval_equals_standalone():
    """A coded-diffraction request served beside MaxCut requests runs on its own
    graphs: its objective and infeasibility equal the standalone handle's bit
    for bit, and the MaxCut requests of the same rounds are unaffected."""
    from paper_1912_02949_gb300 import scgal as S
    S.load()
    n, L, T = 1024, 5, 40
    pd = W.phase_problem(n, L, seed=0)
    p = S.scgal_params_default(R=5, T_max=T, precision=32)
    h = S.scgal_create_phase(pd.masks, L, n, pd.b, 0.0, p)
    rc, last = S.scgal_solve(h, T)
    _, lam, _, _ = S.scgal_reconstruct(h, want_cut=False)
    h.close()
    g = W.er_graph(2000, 8000, seed=3, weights="unit")
    rp, col, _ = g.csr()
    pm = S.scgal_params_default(R=10, T_max=30, precision=32)
    alone = S.scgal_server_create(1 << 32, 4)
    ref_mc = S.scgal_poll(alone, S.scgal_submit(alone, rp, col, None, g.n, col.size, pm), -1)
    S.scgal_server_destroy(alone)
    srv = S.scgal_server_create(1 << 32, 4)
    t_mc = S.scgal_submit(srv, rp, col, None, g.n, col.size, pm)
    t_ph = S.scgal_submit_phase(srv, pd.masks, L, n, pd.b, p)
    res_ph = S.scgal_poll(srv, t_ph, -1)
    res_mc = S.scgal_poll(srv, t_mc, -1)
    S.scgal_server_destroy(srv)
    assert res_ph["status"] == S.SCGAL_ENOTDONE and res_ph["iterations"] == T and res_ph["n"] == n
    assert res_ph["objective"] == last["p"] and res_ph["infeas"] == last["infeas"]
    assert res_ph["best_cut"] == 0 and abs(res_ph["lambda_max"] - lam[0]) <= 1e-6 * lam[0]
    assert _result_fields(res_mc) == _result_fields(ref_mc)
