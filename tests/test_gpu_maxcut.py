"""GPU parity of the MaxCut path against the FP64 oracle, through the C ABI.

Tolerances (relative): single D-matvec 1e-5 (FP32 path) / 1e-12 (FP64 path);
Lanczos Ritz value on a well-separated spectrum 1e-4 / 1e-10; end-of-run
objective after T iterations 1e-3; end-of-run infeasibility, gap, top
eigenvalue and rounded cut within the oracle's own spread under rounding-level
perturbations of its random draws (the trajectory past the first iterations is
decided by rounding); cut values exact integers for the same sign vector.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.lanczos import approx_min_evec, lanczos_steps
from oracle.nystrom import NystromSketch
from oracle.philox import PURPOSE_LANCZOS, PURPOSE_OMEGA, gaussian_matrix, gaussian_vector
from oracle.problems import MaxCutProblem
from oracle.rounding import cut_weight, round_maxcut
from oracle.sketchycgal import sketchy_cgal

pytestmark = pytest.mark.gpu

TOL_MV = {32: 1e-5, 64: 1e-12}
TOL_XI = {32: 1e-4, 64: 1e-10}


@pytest.fixture(scope="module")
def S():
    from paper_1912_02949_gb300 import build, scgal
    build.build()
    scgal.load()
    return scgal


def _handle(S, g, prec, R=10, T_max=100, seed=0, **kw):
    rp, col, val = g.csr()
    w = None if g.weight_kind == "unit" else val
    p = S.scgal_params_default(R=R, T_max=T_max, precision=prec, seed=seed, **kw)
    return S.scgal_create_maxcut(rp, col, w, g.n, col.size, 0.0, p)


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


GRAPHS = {
    "er_unit": lambda: W.er_graph(3000, 12000, seed=1, weights="unit"),
    "er_pm1": lambda: W.er_graph(5000, 15000, seed=2, weights="pm1"),
    "er_real": lambda: W.er_graph(2000, 9000, seed=3, weights="real"),
    "dense_rows": lambda: W.er_graph(300, 20000, seed=4, weights="pm1"),     # degree ~130: 32-lane rows
    "torus": lambda: W.torus_longrange_graph(32, 64, 0.1, seed=5, weights="pm1"),
}


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("gname", sorted(GRAPHS))
def test_apply_D_matches_oracle(S, gname, prec):
    g = GRAPHS[gname]()
    h = _handle(S, g, prec)
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    r = np.random.default_rng(7)
    x = r.standard_normal(g.n)
    w = 0.01 * r.standard_normal(g.n)
    yg = S.scgal_apply_D(h, x, w)
    yo = prob.C_apply(x) + prob.Astar_apply(w, x)
    assert _relerr(yg, yo) <= TOL_MV[prec]
    assert np.max(np.abs(yg - yo)) <= TOL_MV[prec] * np.max(np.abs(yo))
    info = S.scgal_get_info(h)
    assert info["weight_kind"] == {"unit": 0, "pm1": 1, "real": 2}[g.weight_kind]
    assert math.isclose(info["normC"], prob.normC, rel_tol=1e-12)


@pytest.mark.parametrize("prec", [32, 64])
def test_apply_D_edge_cases(S, prec):
    # isolated vertices and a ragged tail of empty rows
    g = W.er_graph(1000, 300, seed=9, weights="pm1")
    h = _handle(S, g, prec)
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    x = np.random.default_rng(1).standard_normal(g.n)
    w = np.linspace(-1, 1, g.n)
    assert _relerr(S.scgal_apply_D(h, x, w), prob.C_apply(x) + prob.Astar_apply(w, x)) <= TOL_MV[prec]
    # empty graph (C = 0): D = diag(w);  smallest instance n = 2
    for n, m in ((50, 0), (2, 1)):
        g2 = W.er_graph(n, m, seed=0, weights="unit")
        h2 = _handle(S, g2, prec, R=min(10, n))
        p2 = MaxCutProblem(g2.n, g2.i, g2.j, g2.w)
        x2 = np.arange(1.0, n + 1)
        w2 = np.cos(np.arange(n))
        assert _relerr(S.scgal_apply_D(h2, x2, w2), p2.C_apply(x2) + p2.Astar_apply(w2, x2)) <= TOL_MV[prec]


def test_malformed_csr_is_rejected(S):
    p = S.scgal_params_default(T_max=10, R=2)
    rp = np.array([0, 2, 1, 3], dtype=np.int32)          # decreasing row pointer
    col = np.array([1, 2, 0], dtype=np.int32)
    with pytest.raises(S.ScgalError) as e:
        S.scgal_create_maxcut(rp, col, None, 3, 3, 0.0, p)
    assert e.value.status == S.SCGAL_EINVAL
    rp = np.array([0, 1, 2, 3], dtype=np.int32)
    for badcol in ([1, 7, 0], [0, 2, 1]):                 # out of range / diagonal entry
        with pytest.raises(S.ScgalError):
            S.scgal_create_maxcut(rp, np.array(badcol, dtype=np.int32), None, 3, 3, 0.0, p)
    with pytest.raises(S.ScgalError):
        S.scgal_create_maxcut(rp, np.array([1, 2, 0], dtype=np.int32), np.array([1.0, np.nan, 1.0]), 3, 3, 0.0, p)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("q", [1, 7, 40])
def test_lanczos_matches_oracle(S, prec, q):
    g = W.er_graph(4000, 14000, seed=11, weights="pm1")
    h = _handle(S, g, prec, T_max=10 ** 6)
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    r = np.random.default_rng(3)
    w = 0.02 * r.standard_normal(g.n) - 0.01
    t = 5
    xi_g, k, v_g = S.scgal_lanczos(h, t, q, w)
    v1 = gaussian_vector(0, PURPOSE_LANCZOS, t, 0, g.n, False)
    xi_o, v_o, info = approx_min_evec(lambda u: prob.C_apply(u) + prob.Astar_apply(w, u), v1, q)
    assert k == info["k"] == q
    assert abs(xi_g - xi_o) <= TOL_XI[prec] * abs(xi_o)
    v_o = v_o / np.linalg.norm(v_o)
    assert abs(np.linalg.norm(v_g) - 1.0) < 1e-6
    # the Ritz vectors agree up to sign
    assert abs(abs(np.dot(v_g, v_o)) - 1.0) <= (1e-3 if prec == 32 else 1e-9)


def _oracle_ensemble(prob, R, T, seed, eps, runs=8):
    """The oracle rerun with its random start vectors perturbed by `eps` relative
    (1e-16 for the FP64 path, 1e-7 for the FP32 path): the spread of its own
    end-of-run values under rounding-level changes.  Past the first iterations the
    Lanczos runs lose orthogonality (an outlier Ritz value converges within a few
    steps once v_1 has localised) and the trajectory depends on rounding, so only
    quantities that are stable under this ensemble can be compared."""
    import oracle.sketchycgal as SC
    orig = SC.gaussian_vector
    out = []
    try:
        for k in range(runs):
            rng = np.random.default_rng(1000 + k)
            e = 0.0 if k == 0 else eps
            SC.gaussian_vector = lambda *a, e=e, rng=rng, **kw: (lambda v: v * (1 + e * rng.standard_normal(v.shape)))(orig(*a, **kw))
            out.append(SC.sketchy_cgal(prob, R=R, T=T, seed=seed))
    finally:
        SC.gaussian_vector = orig
    return out


def _within_ensemble(x, vals, floor):
    """x lies in the ensemble's range widened by 1.5 times its spread (and an absolute floor)."""
    lo, hi = min(vals), max(vals)
    pad = max(1.5 * (hi - lo), floor)
    return lo - pad <= x <= hi + pad


@pytest.mark.parametrize("prec", [32, 64])
def test_end_to_end_er800(S, prec):
    """The n = 800, 19,176-edge Erdos-Renyi MaxCut SDP (smallest Gset shape), T = 500."""
    g = W.config_graph("er800")
    T = 500
    h = _handle(S, g, prec, R=10, T_max=T)
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    ens = _oracle_ensemble(prob, R=10, T=T, seed=0, eps=1e-7 if prec == 32 else 1e-16)
    ref = ens[0]
    rc, last = S.scgal_solve(h, T)
    assert rc == S.SCGAL_ENOTDONE and last["t"] == T
    hist = S.scgal_history(h, 1, T)
    assert [r["q"] for r in hist] == [r["q"] for r in ref.history]
    # the well-conditioned start of the trajectory is reproduced step for step
    # (FP32: only t = 1; at t = 2 an FP32 Lanczos run's xi already spreads by ~3%
    # under 1e-7 perturbations, because D_2 has an outlier eigenvalue)
    for rg, rr in zip(hist[:(1 if prec == 32 else 3)], ref.history[:3]):
        assert abs(rg["xi"] - rr["xi"]) <= TOL_XI[prec] * abs(rr["xi"])
        assert abs(rg["p"] - rr["p_orig"]) <= TOL_XI[prec] * max(abs(rr["p_orig"]), 1.0)
    # end of run: objective within 1e-3 relative
    ro = ref.history[-1]
    assert abs(last["p"] - ro["p_orig"]) <= 1e-3 * abs(ro["p_orig"])
    # infeasibility and gap: inside the oracle's own rounding spread
    assert _within_ensemble(last["infeas"], [e.history[-1]["infeas"] for e in ens], 1e-3)
    assert _within_ensemble(last["relgap"], [e.history[-1]["relgap"] for e in ens], 1e-3)
    U, lam, err, cut = S.scgal_reconstruct(h)
    assert math.isclose(lam.sum(), ref.Lam.sum(), rel_tol=1e-9)       # trace correction: tr = alpha
    assert _within_ensemble(lam[0], [e.Lam[0] for e in ens], 1e-3 * lam[0])
    # the GPU's cut is exactly the oracle's evaluation of the GPU's sign vectors
    best, col, cuts = round_maxcut(U.T, g.i, g.j, g.w)
    assert cut == best
    cuts_o = [round_maxcut(e.U, g.i, g.j, g.w)[0] for e in ens]
    assert _within_ensemble(cut, cuts_o, 0.005 * cuts_o[0])


def test_cut_value_exact(S):
    for weights in ("unit", "pm1"):
        g = W.er_graph(20000, 70000, seed=21, weights=weights)
        h = _handle(S, g, 32)
        r = np.random.default_rng(5)
        for _ in range(3):
            chi = np.where(r.random(g.n) < 0.5, -1, 1).astype(np.int8)
            assert S.scgal_cut_value(h, chi) == cut_weight(g.i, g.j, g.w, chi)


@pytest.mark.parametrize("prec", [32, 64])
def test_nystrom_reconstruct_matches_oracle(S, prec):
    """Alg. B.1 on a planted rank-3 psd X with the handle's own Omega."""
    n, R = 3000, 8
    g = W.er_graph(n, 9000, seed=2, weights="unit")
    h = _handle(S, g, prec, R=R, scale=0)       # unscaled: alpha = n, no X scaling on output
    Om = gaussian_matrix(0, PURPOSE_OMEGA, 0, n, R, False)
    if prec == 32:
        Om = Om.astype(np.float32).astype(np.float64)
    r = np.random.default_rng(4)
    Q, _ = np.linalg.qr(r.standard_normal((n, 3)))
    ev = np.array([500.0, 200.0, 100.0])
    Sk = (Q * ev) @ (Q.T @ Om)
    tau = float(ev.sum())
    S.scgal_set_state(h, S=Sk, tau=tau, t=1)
    sk = NystromSketch(Om)
    sk.S = Sk.astype(np.float32).astype(np.float64) if prec == 32 else Sk
    sk.tau = tau
    Uo, Lo, eo = sk.reconstruct()
    U, lam, err, _ = S.scgal_reconstruct(h, want_cut=False)
    # the trace correction (default on for MaxCut) shifts all R values by (alpha - tr)/R
    shift = (n - Lo.sum()) / R
    tol = 1e-4 if prec == 32 else 1e-8
    np.testing.assert_allclose(lam[:3] - shift, Lo[:3], rtol=tol)
    np.testing.assert_allclose(err[:3], eo[:3], rtol=tol, atol=tol * tau)
    for c in range(3):
        assert abs(abs(np.dot(U[c], Uo[:, c])) - 1.0) <= tol


def test_checkpoint_resume_is_bitwise(S):
    g = W.er_graph(3000, 10000, seed=8, weights="pm1")
    a = _handle(S, g, 32, T_max=60)
    S.scgal_solve(a, 30)
    st = S.scgal_get_state(a)
    S.scgal_solve(a, 50)
    ra = S.scgal_history(a, 31, 20)
    b = _handle(S, g, 32, T_max=60)
    S.scgal_set_state(b, z=st["z"], y=st["y"], S=st["S"], p=st["p"], tau=st["tau"], t=st["t"])
    S.scgal_solve(b, 50)
    rb = S.scgal_history(b, 31, 20)
    assert ra == rb


def test_stopping_rule_and_state_errors(S):
    g = W.cycle_graph(8)
    h = _handle(S, g, 64, R=4, T_max=5000, tol=1e-3)
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    ref = sketchy_cgal(prob, R=4, T=5000, seed=0, tol=1e-3)
    rc, last = S.scgal_solve(h, 5000)
    assert rc == S.SCGAL_OK and last["converged"] == 1
    assert abs(last["t"] - ref.converged_at) <= 2
    assert last["relgap"] <= 1e-3 and last["infeas"] <= 1e-3
    with pytest.raises(S.ScgalError) as e:
        S.scgal_step(h)
    assert e.value.status == S.SCGAL_ESTATE


def test_full_size_er2p20_matvec_and_first_iterations(S):
    """n = 2^20, m = 3n, +/-1 weights (the bench workload) in the bench's launch
    shape: one D-matvec, the first iteration against the oracle, then the exact
    invariant sum(z) = tau = tr X' of the following iterations (the trajectory
    itself depends on rounding from t = 2 on: D_2 has an outlier eigenvalue that
    Lanczos converges to, which destroys orthogonality)."""
    g = W.config_graph("er2p20")
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    r = np.random.default_rng(0)
    x = r.standard_normal(g.n)
    w = 1e-3 * r.standard_normal(g.n)
    yo = prob.C_apply(x) + prob.Astar_apply(w, x)
    ref = sketchy_cgal(prob, R=10, T=1, seed=0)
    for prec in (32, 64):
        h = _handle(S, g, prec, R=10, T_max=2000)
        yg = S.scgal_apply_D(h, x, w)
        assert _relerr(yg, yo) <= TOL_MV[prec]
        S.scgal_step(h)
        st = S.scgal_get_state(h)
        assert _relerr(st["z"], ref.z) <= (1e-4 if prec == 32 else 1e-10)
        assert _relerr(st["y"], ref.y) <= (1e-4 if prec == 32 else 1e-10)
        assert abs(st["p"] - ref.p) <= (1e-4 if prec == 32 else 1e-10) * abs(ref.p)
        S.scgal_solve(h, 6)
        st = S.scgal_get_state(h)
        assert math.isclose(st["z"].sum(), st["tau"], rel_tol=(1e-5 if prec == 32 else 1e-12))
        assert math.isclose(st["tau"], 1.0, rel_tol=1e-12)      # every step took H = v v*: tr X' = 1
        h.close()


def test_full_size_torus2p23_matvec_and_first_iteration(S):
    """n = 2^23: 2048 x 4096 torus plus 10% long-range edges, +/-1 weights (the
    largest MaxCut workload; basis and sketch resident on one GPU).  One D-matvec
    against the oracle; the first iteration's z = A(v v*) = |v|^2 (eta_1 = 1)
    against the oracle's ApproxMinEvec on the same start vector; then the exact
    invariant sum(z) = tau = tr X' = 1 after a few more iterations."""
    g = W.config_graph("torus2p23")
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    h = _handle(S, g, 32, R=10, T_max=1000)
    r = np.random.default_rng(2)
    x = r.standard_normal(g.n)
    w = 1e-4 * r.standard_normal(g.n)
    assert _relerr(S.scgal_apply_D(h, x, w), prob.C_apply(x) + prob.Astar_apply(w, x)) <= TOL_MV[32]
    S.scgal_step(h)
    st = S.scgal_get_state(h)
    w1 = -math.sqrt(2) * prob.b                       # y = z = 0 at t = 1
    v1 = gaussian_vector(0, PURPOSE_LANCZOS, 1, 0, g.n, False)
    _, v, _ = approx_min_evec(lambda u: prob.C_apply(u) + prob.Astar_apply(w1, u), v1, lanczos_steps(g.n, 1))
    z_ref = (v / np.linalg.norm(v)) ** 2
    assert _relerr(st["z"], z_ref) <= 1e-4
    S.scgal_solve(h, 4)
    st = S.scgal_get_state(h)
    assert math.isclose(st["z"].sum(), st["tau"], rel_tol=1e-5)
    assert math.isclose(st["tau"], 1.0, rel_tol=1e-12)
    h.close()


def test_autotuned_grid_is_cached_and_leaves_the_state_alone(S):
    """params.tune: the first handle times the candidate D-matvec grids (on its
    own graph, private scalars) and caches the pick; a second handle of the same
    shape reuses it without running the tuning launches.  Identical histories
    show that the tuning launches did not disturb the first handle's state; the
    tuned D-matvec matches the oracle like the fixed shape."""
    g = W.er_graph(20000, 80000, seed=9, weights="pm1")
    T = 40
    a = _handle(S, g, 32, T_max=T, tune=1)
    b = _handle(S, g, 32, T_max=T, tune=1)
    ia, ib = S.scgal_get_info(a), S.scgal_get_info(b)
    assert ia["spmv_grid"] == ib["spmv_grid"] > 0
    S.scgal_solve(a, T)
    S.scgal_solve(b, T)
    assert S.scgal_history(a, 1, T) == S.scgal_history(b, 1, T)
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    r = np.random.default_rng(2)
    x = r.standard_normal(g.n)
    w = r.standard_normal(g.n)
    yo = prob.C_apply(x) + prob.Astar_apply(w, x)
    assert _relerr(S.scgal_apply_D(b, x, w), yo) <= TOL_MV[32]
