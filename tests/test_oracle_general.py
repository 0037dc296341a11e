"""Pins for the oracle's general template (Alg. D.1, App. D.3 item 1): the
inclusion A(X) in K = {u : u <= b} through the slack w = proj_K(z + y/beta).

* The projection against its definition (nearest point of K, sampled).
* Inactive constraints (b far above any reachable A(X)): the slack absorbs
  z + y/beta, so y stays exactly 0, D = C every iteration, and the method is
  Frank-Wolfe on <C, X> over alpha Delta: p_T -> alpha lambda_min(C).
* MaxCut with diag X <= 1 (tr X <= n): against the SDP value certified by an
  independent solver (projected gradient on the Burer-Monteiro factor with a
  dual certificate C + diag(y) >= 0), on +/-1-weighted graphs where some rows
  are slack at the optimum; against the closed form n^2/4 of the complete graph
  (the Laplacian is psd, so raising a diagonal entry never lowers tr(LX): the
  optimum has diag X = 1 and equals Eq. 1.2's); and the all-negative-weight
  graph, whose optimum X = 0 leaves every constraint slack.
* The derived stopping bound p - p* <= p + <y,w> + beta/2 <z-w, z+w> - alpha
  min(0, lambda_min(D)) on the final state, with the exact lambda_min.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.problems import MaxCutProblem
from oracle.sketchycgal import al_weights, proj_K, sketchy_cgal, stopping_values


def test_projection_is_the_nearest_point_of_K():
    r = np.random.default_rng(0)
    for _ in range(20):
        b = r.standard_normal(7)
        w = 2.0 * r.standard_normal(7)
        pw = proj_K(w, b, "leq")
        assert np.all(pw <= b)
        for _ in range(200):                       # any other point of K is no closer
            u = b - np.abs(r.standard_normal(7)) * r.exponential(1.0, 7)
            assert np.linalg.norm(w - pw) <= np.linalg.norm(w - u) + 1e-15
        # and no point of K near pw is closer either (local optimality, all directions)
        for _ in range(200):
            u = np.minimum(pw + 1e-3 * r.standard_normal(7), b)
            assert np.linalg.norm(w - pw) <= np.linalg.norm(w - u) + 1e-15
    assert np.array_equal(proj_K(w, b, "eq"), b)


def test_weights_are_the_gradient_of_the_slack_augmented_lagrangian():
    """u = y + beta (z - proj_K(z + y/beta)) is the gradient in z of
    phi(z) = min over w in K of <y, z - w> + beta/2 ||z - w||^2 (so D = C + A*(u)
    is the derivative of the augmented Lagrangian of App. D.4 in X); the inner
    minimum is solved numerically under the bound w <= b, the gradient by
    central differences."""
    from scipy.optimize import minimize
    r = np.random.default_rng(3)
    d = 6
    for _ in range(5):
        z, y, b = r.standard_normal(d), r.standard_normal(d), 0.3 * r.standard_normal(d)
        beta = float(r.uniform(0.5, 3.0))

        def phi(zz):
            f = lambda w: float(np.dot(y, zz - w) + 0.5 * beta * np.dot(zz - w, zz - w))
            g = lambda w: -y - beta * (zz - w)
            best = min((minimize(f, w0, jac=g, method="L-BFGS-B", bounds=[(None, bi) for bi in b],
                                 options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 2000})
                        for w0 in (np.minimum(zz, b), b - 1.0)), key=lambda o: o.fun)
            return best.fun

        h = 1e-5
        fd = np.array([(phi(z + h * e) - phi(z - h * e)) / (2 * h) for e in np.eye(d)])
        np.testing.assert_allclose(al_weights(z, y, beta, b, "leq"), fd, rtol=1e-5, atol=1e-6)


def test_gap_numerator_is_surrogate_gap_minus_lagrangian_offset():
    """The stopping numerator equals <D, X> - alpha min(0, xi) - (L(X) - p) with
    <D, X> = p + <u, z>, u the weights, and L(X) - p = <y, z - w> + beta/2 ||z - w||^2,
    the definition it was derived from (any dropped term or sign shows here)."""
    g = W.cycle_graph(7)
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    r = np.random.default_rng(5)
    for _ in range(10):
        z, y = 0.3 * r.random(g.n), r.standard_normal(g.n)
        p, beta, xi = float(r.standard_normal()), float(r.uniform(1, 5)), float(r.standard_normal())
        relgap, _, p_orig = stopping_values(prob, p, y, z, beta, xi, "leq", "leq")
        w = np.minimum(z + y / beta, prob.b)
        u = al_weights(z, y, beta, prob.b, "leq")
        num = (p + float(np.dot(u, z)) - prob.alpha * min(0.0, xi)) \
            - (float(np.dot(y, z - w)) + 0.5 * beta * float(np.dot(z - w, z - w)))
        assert math.isclose(relgap, prob.obj_factor * num / (1.0 + abs(p_orig)), rel_tol=1e-12, abs_tol=1e-12)


def _pm1_graph(n, seed):
    """A connected +/-1-weighted graph on n vertices (a cycle plus random chords)."""
    r = np.random.default_rng(seed)
    edges = {(i, (i + 1) % n) for i in range(n)}
    while len(edges) < 2 * n:
        i, j = sorted(r.choice(n, 2, replace=False))
        edges.add((int(i), int(j)))
    e = np.array(sorted(edges))
    w = np.where(r.random(len(e)) < 0.5, -1.0, 1.0)
    return e[:, 0], e[:, 1], w


def _certified_sdp(C, starts=6, iters=40000):
    """min <C, X> s.t. diag X <= 1, X psd, by projected gradient on X = V V^T
    (rows of V in the unit ball), certified by a dual point: p* >= -sum(y) for
    any y >= 0 with C + diag(y) psd.  Returns (primal value, certified lower bound)."""
    n = C.shape[0]
    r = np.random.default_rng(1)
    step = 0.25 / max(np.abs(np.linalg.eigvalsh(C)).max(), 1e-12)
    best = None
    for _ in range(starts):
        V = r.standard_normal((n, n))
        V /= np.maximum(1.0, np.linalg.norm(V, axis=1))[:, None]
        for _ in range(iters):
            V = V - step * 2.0 * (C @ V)
            V /= np.maximum(1.0, np.linalg.norm(V, axis=1))[:, None]
        f = float(np.sum(C * (V @ V.T)))
        if best is None or f < best[0]:
            best = (f, V)
    f, V = best
    # KKT multipliers of the rows on the sphere, then shift until C + diag(y) is psd
    rn2 = np.sum(V * V, axis=1)
    y = np.where(rn2 > 1.0 - 1e-9, -np.sum((C @ V) * V, axis=1) / np.maximum(rn2, 1e-300), 0.0)
    y = np.maximum(y, 0.0)
    lam = np.linalg.eigvalsh(C + np.diag(y))[0]
    y = y + max(0.0, -lam)
    return f, -float(np.sum(y))


def _run_leq(prob, T, R=4):
    return sketchy_cgal(prob, R=R, T=T, seed=0, kset="leq", lmo="leq")


def test_inactive_constraints_reduce_to_frank_wolfe_on_C():
    g = W.cycle_graph(9)
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    prob.b_orig = 1e6 * np.ones(g.n)             # never reached: A(X) = diag X <= tr X = alpha
    prob._set_scale(True)
    T = 400
    res = sketchy_cgal(prob, R=4, T=T, seed=0, kset="leq")
    assert np.all(res.y == 0.0)
    assert all(h["gamma"] == 1.0 for h in res.history)     # z - wbar = 0: gamma = beta0
    lam = np.linalg.eigvalsh(prob.dense_C())[0]
    # every recorded Ritz value is that of C itself (an upper bound on lambda_min(C))
    assert all(h["xi"] >= lam - 1e-12 for h in res.history)
    assert abs(res.history[-1]["xi"] - lam) <= 1e-9 * abs(lam)
    # Frank-Wolfe with step 2/(t+1) on <C, X> over Delta: p_T within 1e-3 of alpha lambda_min
    assert abs(res.p - prob.alpha * lam) <= 1e-3 * abs(prob.alpha * lam)
    # constraints inactive: distance to K is 0
    assert res.history[-1]["infeas"] == 0.0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_leq_maxcut_matches_certified_sdp(seed):
    n = 8
    i, j, w = _pm1_graph(n, seed)
    prob = MaxCutProblem(n, i, j, w)
    C = -0.25 * prob.L.toarray()
    f, lb = _certified_sdp(C)
    assert f - lb <= 1e-7 * max(1.0, abs(f))      # the independent solver is certified
    pstar = f
    res = _run_leq(prob, T=4000)
    h = res.history[-1]
    assert abs(h["p_orig"] - pstar) <= 1e-2 * max(1.0, abs(pstar))
    assert h["infeas"] <= 1e-2
    # the stopping gap closes at the optimum (it oscillates around 0 by ~1e-2:
    # the inexact xi of the Lanczos run stands in for lambda_min, App. E)
    assert max(abs(r["relgap"]) for r in res.history[-20:]) <= 3e-2
    # the derived bound on the final state, with the exact lambda_min(D)
    t = res.t_done + 1
    beta = math.sqrt(t + 1)
    wk = proj_K(res.z + res.y / beta, prob.b, "leq")
    D = prob.dense_C() + np.diag(prob.sA * (res.y + beta * (res.z - wk)))
    lam = np.linalg.eigvalsh(D)[0]
    num = res.p + float(np.dot(res.y, wk)) + 0.5 * beta * float(np.dot(res.z - wk, res.z + wk)) \
        - prob.alpha * min(0.0, lam)
    assert res.p - pstar / prob.obj_factor <= num + 1e-12


def test_leq_some_rows_slack_at_the_optimum():
    """The +/-1 instances above do exercise the inequality: at the certified
    optimum some diagonal entries are below 1 (else the test would only repeat
    the equality case)."""
    slack = 0
    for seed in range(3):
        i, j, w = _pm1_graph(8, seed)
        prob = MaxCutProblem(8, i, j, w)
        res = _run_leq(prob, T=4000)
        Xd = res.z * prob.z_factor                 # diag X = A(X) in the original units
        slack += int(np.sum(Xd < 0.9))
    assert slack > 0


@pytest.mark.parametrize("n", [6, 7])
def test_leq_complete_graph_closed_form(n):
    g = W.complete_graph(n)
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    res = _run_leq(prob, T=3000)
    h = res.history[-1]
    assert abs(-h["p_orig"] - n * n / 4.0) <= 2e-3 * n * n / 4.0
    assert h["infeas"] <= 1e-2


def test_leq_all_negative_weights_optimum_is_zero():
    n = 8
    i, j, _ = _pm1_graph(n, 3)
    prob = MaxCutProblem(n, i, j, -np.ones(i.size))
    res = _run_leq(prob, T=500)
    h = res.history[-1]
    assert abs(h["p_orig"]) <= 1e-3 * n
    assert h["infeas"] == 0.0
