"""Pins for the oracle's ApproxMinEvec (Alg. 4.1) against a dense eigensolver."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.lanczos import approx_min_evec, lanczos_steps, tridiag_min_eig
from oracle.philox import PURPOSE_LANCZOS, gaussian_vector
from oracle.problems import MaxCutProblem, PhaseProblem


def _gradient(prob, seed=0):
    """A gradient D = C + A*(w) of the kind SketchyCGAL forms (Eq. 6.1)."""
    r = np.random.default_rng(seed)
    w = 0.1 * r.standard_normal(prob.d)
    Mv = lambda u: prob.C_apply(u) + prob.Astar_apply(w, u)
    n = prob.n
    E = np.eye(n, dtype=np.complex128 if prob.complex_ else np.float64)
    M = np.stack([Mv(E[:, k]) for k in range(n)], axis=1)
    return Mv, M


def test_q_rule():
    assert lanczos_steps(800, 1) == math.ceil(math.log(800))
    assert lanczos_steps(1 << 20, 2000) == 93
    assert lanczos_steps(5, 10 ** 6) == 4  # capped at n - 1


@pytest.mark.parametrize("kind", ["maxcut", "phase"])
def test_full_krylov_space_gives_exact_min_eigenpair(kind):
    """With q >= n-1 the Krylov space is everything: xi = lambda_min(M)."""
    if kind == "maxcut":
        g = W.er_graph(60, 200, seed=4, weights="pm1")
        prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    else:
        pd = W.phase_problem(16, 12, seed=4)
        prob = PhaseProblem(pd.masks, pd.b)
    Mv, M = _gradient(prob)
    lam, V = np.linalg.eigh(M)
    v1 = gaussian_vector(0, PURPOSE_LANCZOS, 1, 0, prob.n, prob.complex_)
    # full reorthogonalisation is not part of Alg. 4.1, so give it room: q = 3n
    xi, v, info = approx_min_evec(Mv, v1, 3 * prob.n)
    assert info["k"] <= prob.n - 1 or info["k"] == prob.n - 1
    assert abs(xi - lam[0]) <= 1e-9 * np.max(np.abs(lam))
    v = v / np.linalg.norm(v)
    rq = np.real(np.vdot(v, M @ v))
    assert abs(rq - lam[0]) <= 1e-7 * np.max(np.abs(lam))


def test_tridiagonal_matches_dense_projection():
    """T built by the recurrence equals V* M V for the Lanczos basis, and xi is
    its minimum eigenvalue (dense check of the three-term recurrence)."""
    g = W.er_graph(120, 500, seed=5, weights="unit")
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    Mv, M = _gradient(prob, 1)
    v1 = gaussian_vector(3, PURPOSE_LANCZOS, 1, 0, prob.n, False)
    q = 12
    # explicit Gram-Schmidt Krylov basis, independent of the recurrence
    K = [v1 / np.linalg.norm(v1)]
    for _ in range(q - 1):
        x = M @ K[-1]
        for b in K:
            x = x - np.dot(b, x) * b
        K.append(x / np.linalg.norm(x))
    Q = np.stack(K, axis=1)
    Tdense = Q.T @ M @ Q
    xi, v, info = approx_min_evec(Mv, v1, q)
    np.testing.assert_allclose(info["omegas"], np.diag(Tdense), rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(info["rhos"], np.abs(np.diag(Tdense, 1)), rtol=1e-8, atol=1e-12)
    assert math.isclose(xi, np.linalg.eigvalsh(Tdense)[0], rel_tol=1e-10)


def test_tridiag_min_eig_small_cases():
    assert tridiag_min_eig([3.0], []) == (3.0, np.ones(1)) or tridiag_min_eig([3.0], [])[0] == 3.0
    xi, u = tridiag_min_eig([2.0, 2.0], [1.0])
    assert math.isclose(xi, 1.0, rel_tol=1e-14)
    np.testing.assert_allclose(np.abs(u), [1 / math.sqrt(2)] * 2, rtol=1e-12)


def test_store_and_regenerate_agree():
    g = W.er_graph(200, 900, seed=6, weights="pm1")
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    Mv, _ = _gradient(prob, 2)
    v1 = gaussian_vector(1, PURPOSE_LANCZOS, 9, 0, prob.n, False)
    xa, va, _ = approx_min_evec(Mv, v1, 20, store_basis=True)
    xb, vb, _ = approx_min_evec(Mv, v1, 20, store_basis=False)
    assert xa == xb
    np.testing.assert_allclose(va, vb, rtol=1e-12, atol=1e-14)


def test_breakdown_on_invariant_subspace():
    """Start vector = eigenvector: v_2 = M v_1 - omega_1 v_1 is exactly 0, so the
    loop breaks with rho_1 = 0 and T is 1 x 1 (the exact test of Alg. 4.1)."""
    n = 50
    D = np.diag(np.arange(n, dtype=float) - 7.0)
    v1 = np.zeros(n)
    v1[9] = 3.0
    xi, v, info = approx_min_evec(lambda u: D @ u, v1, 10)
    assert info["k"] == 1
    assert xi == 2.0
    np.testing.assert_array_equal(v, v1 / 3.0)


def test_randomized_lanczos_error_bound():
    """Fact 4.1: with q >= 1/2 + eps^{-1/2} log(n / delta^2), the Ritz vector
    satisfies u*Mu <= lambda_min + (eps/8) ||M|| with probability >= 1 - 2 delta."""
    g = W.er_graph(150, 700, seed=7, weights="pm1")
    prob = MaxCutProblem(g.n, g.i, g.j, g.w)
    Mv, M = _gradient(prob, 3)
    lam = np.linalg.eigvalsh(M)
    normM = np.max(np.abs(lam))
    eps, delta = 0.5, 0.1
    q = math.ceil(0.5 + eps ** -0.5 * math.log(prob.n / delta ** 2))
    ok = 0
    trials = 300
    for s in range(trials):
        v1 = gaussian_vector(11, PURPOSE_LANCZOS, s + 1, 0, prob.n, False)
        _, v, _ = approx_min_evec(Mv, v1, q)
        v = v / np.linalg.norm(v)
        ok += (v @ M @ v) <= lam[0] + eps / 8 * normM
    assert ok / trials >= 1 - 2 * delta
