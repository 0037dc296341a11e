"""GPU parity of the general template (Alg. D.1) with inequality constraints,
K = {u : u <= b} (App. D.3 item 1), against the FP64 oracle, through the C ABI.

MaxCut with diag X <= 1 and tr X <= n on +/-1-weighted graphs (rows with a
negative weighted degree are slack at the optimum).  Tolerances as for the
equality path (test_gpu_maxcut): the first iterations step for step (1e-10
FP64, 1e-4 FP32), the end-of-run objective within 1e-3, infeasibility and gap
within the oracle's own spread under rounding-level perturbations; on an
8-vertex graph the GPU reaches the SDP value certified by an independent
solver (tests/test_oracle_general.py).
"""
import numpy as np
import pytest

import workloads as W
from oracle.problems import MaxCutProblem, PhaseProblem
from oracle.sketchycgal import sketchy_cgal

pytestmark = pytest.mark.gpu

TOL_XI = {32: 1e-4, 64: 1e-10}


@pytest.fixture(scope="module")
def S():
    from paper_1912_02949_gb300 import build, scgal
    build.build()
    scgal.load()
    return scgal


def _leq_handle(S, g, prec, R=10, T_max=100, **kw):
    rp, col, val = g.csr()
    w = None if g.weight_kind == "unit" else val
    p = S.scgal_params_default(R=R, T_max=T_max, precision=prec, kset=S.SCGAL_K_LEQ, lmo=S.SCGAL_LMO_LEQ, **kw)
    return S.scgal_create_maxcut(rp, col, w, g.n, col.size, 0.0, p)


def _ensemble(prob, R, T, eps, runs=4, **kw):
    """The oracle rerun with its Lanczos starts perturbed by eps relative (see
    test_gpu_maxcut._oracle_ensemble): the spread of its end-of-run values."""
    import oracle.sketchycgal as SC
    orig = SC.gaussian_vector
    out = []
    try:
        for k in range(runs):
            rng = np.random.default_rng(2000 + k)
            e = 0.0 if k == 0 else eps
            SC.gaussian_vector = lambda *a, e=e, rng=rng, **k2: (lambda v: v * (1 + e * rng.standard_normal(v.shape)))(orig(*a, **k2))
            out.append(SC.sketchy_cgal(prob, R=R, T=T, seed=0, **kw))
    finally:
        SC.gaussian_vector = orig
    return out


def _within(x, vals, floor):
    lo, hi = min(vals), max(vals)
    pad = max(1.5 * (hi - lo), floor)
    return lo - pad <= x <= hi + pad


@pytest.mark.parametrize("prec", [32, 64])
def test_leq_maxcut_er800_matches_oracle(S, prec):
    g = W.er_graph(800, 19176, seed=0, weights="pm1")
    T = 400
    h = _leq_handle(S, g, prec, T_max=T)
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    ens = _ensemble(prob, 10, T, 1e-7 if prec == 32 else 1e-16, kset="leq", lmo="leq")
    ref = ens[0]
    rc, last = S.scgal_solve(h, T)
    assert rc == S.SCGAL_ENOTDONE and last["t"] == T
    hist = S.scgal_history(h, 1, T)
    assert [r["q"] for r in hist] == [r["q"] for r in ref.history]
    for rg, rr in zip(hist[:(1 if prec == 32 else 3)], ref.history[:3]):
        assert abs(rg["xi"] - rr["xi"]) <= TOL_XI[prec] * abs(rr["xi"])
        assert abs(rg["p"] - rr["p_orig"]) <= TOL_XI[prec] * max(abs(rr["p_orig"]), 1.0)
        assert abs(rg["relgap"] - rr["relgap"]) <= TOL_XI[prec] * max(abs(rr["relgap"]), 1.0)
        assert abs(rg["infeas"] - rr["infeas"]) <= TOL_XI[prec] * max(abs(rr["infeas"]), 1e-3)
        assert abs(rg["gamma"] - rr["gamma"]) <= TOL_XI[prec] * abs(rr["gamma"])
    ro = ref.history[-1]
    assert abs(last["p"] - ro["p_orig"]) <= 1e-3 * abs(ro["p_orig"])
    assert _within(last["infeas"], [e.history[-1]["infeas"] for e in ens], 1e-3)
    assert _within(last["relgap"], [e.history[-1]["relgap"] for e in ens], 1e-3)
    # rows with diag X well below 1: the inequality is doing something here
    st = S.scgal_get_state(h)
    assert np.sum(st["z"] * prob.z_factor < 0.9) > 0


def test_leq_maxcut_certified_small_graph(S):
    """8 vertices, +/-1 weights: the FP64 GPU solve against the oracle's
    trajectory and the SDP value certified in the oracle pins."""
    from test_oracle_general import _certified_sdp, _pm1_graph
    i, j, w = _pm1_graph(8, 0)
    g = W.Graph(8, i, j, w, "pm1")
    prob = MaxCutProblem(8, i, j, w)
    f, lb = _certified_sdp(-0.25 * prob.L.toarray())
    T = 4000
    h = _leq_handle(S, g, 64, R=4, T_max=T)
    rc, last = S.scgal_solve(h, T)
    ref = sketchy_cgal(prob, R=4, T=T, seed=0, kset="leq", lmo="leq").history[-1]
    assert abs(last["p"] - ref["p_orig"]) <= 1e-6 * abs(ref["p_orig"])
    assert abs(last["p"] - f) <= 1e-2 * abs(f)
    assert last["infeas"] <= 1e-2


def test_leq_phase_retrieval_zero_is_optimal(S):
    """|FFT(psi_j .* x)|^2 <= b with C = I: X = 0 is feasible and optimal, and
    the trace-bounded LMO never leaves it (D_t = C' = I / sqrt(n) every step)."""
    n, L, T = 256, 4, 30
    pd = W.phase_problem(n, L, seed=0)
    h = S.scgal_create_phase(pd.masks, L, n, pd.b, 0.0,
                             S.scgal_params_default(R=3, T_max=T, precision=64, kset=S.SCGAL_K_LEQ))
    rc, last = S.scgal_solve(h, T)
    ref = sketchy_cgal(PhaseProblem(pd.masks, pd.b), R=3, T=T, seed=0, kset="leq").history
    hist = S.scgal_history(h, 1, T)
    assert all(r["p"] == 0.0 and r["infeas"] == 0.0 for r in hist)
    for rg, rr in zip(hist, ref):
        assert abs(rg["xi"] - rr["xi"]) <= 1e-10 * abs(rr["xi"])
        assert abs(rg["relgap"] - rr["relgap"]) <= 1e-10 * max(1.0, abs(rr["relgap"]))


def test_leq_served_request_equals_standalone(S):
    """A served K = {u <= b} request runs on its own graphs: bit-identical to
    the standalone handle."""
    g = W.er_graph(3000, 12000, seed=4, weights="pm1")
    rp, col, val = g.csr()
    h = _leq_handle(S, g, 32, T_max=60)
    rc, last = S.scgal_solve(h, 60)
    srv = S.scgal_server_create(1 << 32, 2)
    res = S.scgal_poll(srv, S.scgal_submit(srv, rp, col, val, g.n, col.size,
                                           S.scgal_params_default(R=10, T_max=60, precision=32,
                                                                  kset=S.SCGAL_K_LEQ, lmo=S.SCGAL_LMO_LEQ)), -1)
    S.scgal_server_destroy(srv)
    assert res["iterations"] == 60
    assert res["objective"] == last["p"] and res["infeas"] == last["infeas"]
