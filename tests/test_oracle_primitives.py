"""Pins for the oracle's primitives (Eq. 2.3) and scaling (Eq. 7.1).

The references here are built independently from the definitions: dense
Laplacians from Eq. 1.1, dense measurement matrices A_i = a_i a_i* from an
explicit DFT matrix (App. F.1), numerically computed norms.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle.cgal_dense import dense_maxcut, dense_phase, operator_norm
from oracle.problems import MaxCutProblem, PhaseProblem, PtychoProblem


def _rng(s=0):
    return np.random.default_rng(s)


@pytest.mark.parametrize("weights", ["unit", "pm1", "real"])
@pytest.mark.parametrize("scale", [False, True])
def test_maxcut_primitives_match_dense(weights, scale):
    g = W.er_graph(40, 150, seed=3, weights=weights)
    prob = MaxCutProblem(g.n, g.i, g.j, g.w, scale=scale)
    C, As, b, alpha = dense_maxcut(g.n, g.i, g.j, g.w)
    normC = np.linalg.norm(C, "fro")
    normA = operator_norm(As)
    assert math.isclose(prob.normC, normC, rel_tol=1e-12)
    assert math.isclose(prob.normA, normA, rel_tol=1e-12)
    sC, sA = (1 / normC, 1 / normA) if scale else (1.0, 1.0)
    r = _rng(1)
    u, z = r.standard_normal(g.n), r.standard_normal(g.n)
    np.testing.assert_allclose(prob.C_apply(u), sC * C @ u, rtol=1e-12, atol=1e-12)
    Az = np.einsum("k,kij->ij", z, As)
    np.testing.assert_allclose(prob.Astar_apply(z, u), sA * Az @ u, rtol=1e-12, atol=1e-12)
    Auu = np.array([u @ A @ u for A in As])
    np.testing.assert_allclose(prob.A_of_uu(u), sA * Auu, rtol=1e-12, atol=1e-12)
    if scale:
        np.testing.assert_allclose(prob.b, b / (alpha * normA))
        assert prob.alpha == 1.0


def test_laplacian_quadratic_form_is_cut():
    g = W.er_graph(30, 90, seed=2, weights="pm1")
    prob = MaxCutProblem(g.n, g.i, g.j, g.w, scale=False)
    chi = np.where(_rng(4).standard_normal(g.n) > 0, 1.0, -1.0)
    cut = np.sum(g.w[chi[g.i] != chi[g.j]])
    # chi^T L chi / 4 = weight of the cut (Eq. 1.1 - 1.2)
    assert math.isclose(-chi @ prob.C_apply(chi), cut, abs_tol=1e-9)


@pytest.mark.parametrize("prob_kind", ["maxcut", "phase", "ptycho"])
def test_adjoint_identity(prob_kind):
    """u*(A* z) u = <z, A(u u*)>  (Eq. 2.1).  For ptychography this is the
    identity the Lanczos step's <x, D x> is formed from: sC ||x||^2 plus the
    weighted squared window transforms, without the assembled D x."""
    r = _rng(5)
    if prob_kind == "maxcut":
        g = W.er_graph(64, 300, seed=1, weights="pm1")
        prob = MaxCutProblem(g.n, g.i, g.j, g.w)
        u = r.standard_normal(g.n)
    elif prob_kind == "phase":
        pd = W.phase_problem(32, 12, seed=1)
        prob = PhaseProblem(pd.masks, pd.b)
        u = r.standard_normal(32) + 1j * r.standard_normal(32)
    else:
        pd = W.ptycho_problem(24, 8, 3, seed=1)
        prob = PtychoProblem(24, 8, 3, pd.pupil, pd.b)
        u = r.standard_normal(prob.n) + 1j * r.standard_normal(prob.n)
    z = r.standard_normal(prob.d)
    lhs = np.vdot(u, prob.Astar_apply(z, u))
    rhs = np.dot(z, prob.A_of_uu(u))
    assert abs(lhs.imag) < 1e-9 * abs(rhs)
    assert math.isclose(lhs.real, rhs, rel_tol=1e-12)


def test_fft_primitives_match_naive_dft():
    n, L = 16, 12
    pd = W.phase_problem(n, L, seed=2)
    prob = PhaseProblem(pd.masks, pd.b, scale=False)
    C, As, b, alpha = dense_phase(pd.masks, pd.b)
    r = _rng(6)
    u = r.standard_normal(n) + 1j * r.standard_normal(n)
    z = r.standard_normal(n * L)
    np.testing.assert_allclose(prob.A_of_uu(u), [np.real(np.vdot(u, A @ u)) for A in As], rtol=1e-11)
    np.testing.assert_allclose(prob.Astar_apply(z, u), np.einsum("k,kij->ij", z, As) @ u, rtol=1e-11, atol=1e-9)
    np.testing.assert_allclose(prob.C_apply(u), u)
    # measurements: b = A(chi chi*)  (Eq. 7.2)
    np.testing.assert_allclose(prob.A_of_uu(pd.chi), pd.b, rtol=1e-12)


def test_phase_operator_norm_closed_form():
    """||A|| = n sqrt(L) for unit-modulus masks and the unnormalised DFT."""
    for n in (8, 16):
        pd = W.phase_problem(n, 12, seed=n)
        C, As, b, alpha = dense_phase(pd.masks, pd.b)
        prob = PhaseProblem(pd.masks, pd.b)
        assert math.isclose(operator_norm(As), prob.normA, rel_tol=1e-10)
        assert math.isclose(np.linalg.norm(C, "fro"), prob.normC, rel_tol=1e-12)
        # every ||A_i||_F is equal (= n), as Eq. 7.1 asks
        fro = np.linalg.norm(As.reshape(As.shape[0], -1), axis=1)
        np.testing.assert_allclose(fro, n, rtol=1e-12)


def test_scaled_instance_has_unit_norms():
    g = W.er_graph(24, 60, seed=9, weights="pm1")
    prob = MaxCutProblem(g.n, g.i, g.j, g.w, scale=True)
    C = prob.dense_C()
    assert math.isclose(np.linalg.norm(C, "fro"), 1.0, rel_tol=1e-12)
    E = np.eye(g.n)
    As = np.array([np.diag(prob.A_of_uu(E[:, i])) for i in range(g.n)])
    assert math.isclose(operator_norm(As), 1.0, rel_tol=1e-12)
