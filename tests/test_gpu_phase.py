"""GPU parity of the phase-retrieval path (four-step FFT operators) against the
FP64 oracle (numpy FFT), through the C ABI.  Same tolerances as MaxCut."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.lanczos import approx_min_evec
from oracle.philox import PURPOSE_LANCZOS, gaussian_vector
from oracle.problems import PhaseProblem
from oracle.rounding import phase_error, phase_round
from oracle.sketchycgal import sketchy_cgal

pytestmark = pytest.mark.gpu

TOL_MV = {32: 1e-5, 64: 1e-12}
TOL_XI = {32: 1e-4, 64: 1e-10}
TOL_E2E = {32: 1e-3, 64: 1e-7}


@pytest.fixture(scope="module")
def S():
    from paper_1912_02949_gb300 import build, scgal
    build.build()
    scgal.load()
    return scgal


def _pair(S, n, L, prec, R=5, T_max=100, seed=0, **kw):
    pd = W.phase_problem(n, L, seed=seed)
    h = S.scgal_create_phase(pd.masks, L, n, pd.b, 0.0,
                             S.scgal_params_default(R=R, T_max=T_max, precision=prec, seed=seed, **kw))
    return pd, h, PhaseProblem(pd.masks, pd.b)


def _relerr(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("n,L", [(16, 12), (32, 3), (128, 12), (1024, 5), (1 << 16, 12)])
def test_apply_D_matches_oracle(S, n, L, prec):
    pd, h, prob = _pair(S, n, L, prec)
    r = np.random.default_rng(n)
    x = r.standard_normal(n) + 1j * r.standard_normal(n)
    w = r.standard_normal(L * n)
    yg = S.scgal_apply_D(h, x, w)
    yo = prob.C_apply(x) + prob.Astar_apply(w, x)
    tol = TOL_MV[prec] * (3 if prec == 32 and n >= 1 << 16 else 1)
    assert _relerr(yg, yo) <= tol
    info = S.scgal_get_info(h)
    assert info["is_complex"] == 1 and math.isclose(info["normA"], prob.normA)


def test_invalid_masks_rejected(S):
    pd = W.phase_problem(32, 2, seed=0)
    bad = pd.masks.copy()
    bad[0, 3] = 0.5
    with pytest.raises(S.ScgalError):
        S.scgal_create_phase(bad, 2, 32, pd.b, 0.0, S.scgal_params_default(T_max=5))
    with pytest.raises(S.ScgalError):   # not a power of two
        S.scgal_create_phase(pd.masks[:, :24].copy(), 2, 24, pd.b[:48].copy(), 0.0, S.scgal_params_default(T_max=5))


@pytest.mark.parametrize("prec", [32, 64])
def test_lanczos_matches_oracle(S, prec):
    n, L = 1024, 12
    pd, h, prob = _pair(S, n, L, prec, T_max=1000)
    w = -np.abs(np.random.default_rng(2).standard_normal(L * n)) * 1e-3
    t, q = 4, 25
    xi_g, k, v_g = S.scgal_lanczos(h, t, q, w)
    v1 = gaussian_vector(0, PURPOSE_LANCZOS, t, 0, n, True)
    xi_o, v_o, info = approx_min_evec(lambda u: prob.C_apply(u) + prob.Astar_apply(w, u), v1, q)
    assert k == info["k"]
    assert abs(xi_g - xi_o) <= TOL_XI[prec] * abs(xi_o)
    v_o = v_o / np.linalg.norm(v_o)
    assert abs(abs(np.vdot(v_o, v_g)) - 1.0) <= (1e-3 if prec == 32 else 1e-9)


@pytest.mark.parametrize("prec", [32, 64])
def test_end_to_end_recovers_signal(S, prec):
    n, L, T = 256, 12, 250
    pd, h, prob = _pair(S, n, L, prec, R=5, T_max=T)
    ref = sketchy_cgal(prob, R=5, T=T, seed=0)
    rc, last = S.scgal_solve(h, T)
    ro = ref.history[-1]
    assert abs(last["p"] - ro["p_orig"]) <= TOL_E2E[prec] * abs(ro["p_orig"])
    assert abs(last["infeas"] - ro["infeas"]) <= max(TOL_E2E[prec] * ro["infeas"], 1e-9)
    U, lam, err, _ = S.scgal_reconstruct(h, want_cut=False)
    chi = phase_round(U.T, lam)
    assert phase_error(chi, pd.chi) < 1e-2
    np.testing.assert_allclose(lam[0], ref.Lam[0], rtol=(1e-3 if prec == 32 else 1e-7))


def test_state_roundtrip_in_measurement_order(S):
    n, L = 64, 12
    pd, h, prob = _pair(S, n, L, 64)
    r = np.random.default_rng(1)
    z = r.standard_normal(L * n)
    y = r.standard_normal(L * n)
    S.scgal_set_state(h, z=z, y=y, t=3)
    st = S.scgal_get_state(h)
    np.testing.assert_array_equal(st["z"], z)
    np.testing.assert_array_equal(st["y"], y)
    assert st["t"] == 3


def test_full_size_first_iterations(S):
    """n = 2^16, L = 12 (the abstract phase-retrieval workload): two FP64 iterations."""
    n, L, T = 1 << 16, 12, 2
    pd, h, prob = _pair(S, n, L, 64, R=5, T_max=1000)
    ref = sketchy_cgal(prob, R=5, T=T, seed=0)
    S.scgal_solve(h, T)
    st = S.scgal_get_state(h)
    np.testing.assert_allclose(st["z"], ref.z, rtol=1e-7, atol=1e-12 * np.max(np.abs(ref.z)))
    hist = S.scgal_history(h, 1, T)
    for rg, rr in zip(hist, ref.history):
        assert abs(rg["xi"] - rr["xi"]) <= 1e-9 * abs(rr["xi"])
