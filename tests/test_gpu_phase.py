"""GPU parity of the phase-retrieval path (four-step FFT operators) against the
FP64 oracle (numpy FFT), through the C ABI.  Same tolerances as MaxCut.

The FP32 D-matvec's measured error relative to the oracle (2-norm) is about
1.9e-7 at n = 2^10 and 2.4e-7 at n = 2^16, with 1, 3 or 12 masks alike: the
growth with log2(n) expected of a radix-2 FFT with correctly rounded twiddles,
far inside 1e-5 at every size tested here."""
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
@pytest.mark.parametrize("n,L", [(16, 12), (32, 3), (128, 12), (1024, 5), (1 << 16, 12), (1 << 18, 12), (1 << 20, 3)])
def test_apply_D_matches_oracle(S, n, L, prec):
    pd, h, prob = _pair(S, n, L, prec)
    r = np.random.default_rng(n)
    x = r.standard_normal(n) + 1j * r.standard_normal(n)
    w = r.standard_normal(L * n)
    yg = S.scgal_apply_D(h, x, w)
    yo = prob.C_apply(x) + prob.Astar_apply(w, x)
    assert _relerr(yg, yo) <= TOL_MV[prec]
    assert np.max(np.abs(yg - yo)) <= TOL_MV[prec] * np.max(np.abs(yo))
    info = S.scgal_get_info(h)
    assert info["is_complex"] == 1 and math.isclose(info["normA"], prob.normA)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("n,L", [(256, 3), (1024, 12), (4096, 5), (1 << 14, 12), (1 << 15, 2), (1 << 16, 12),
                                 (1 << 17, 3)])
def test_cluster_kernel_matches_passes_and_oracle(S, n, L, prec):
    """The one-kernel clustered D-matvec (SCGAL_FFT_CLUSTER) against the oracle and
    the three-pass kernels, with the blocks per cluster the library documents."""
    lg = n.bit_length() - 1
    C = 1 << max(0, lg - (13 if prec == 32 else 12))
    fits = C <= 16
    pd = W.phase_problem(n, L, seed=3)
    prob = PhaseProblem(pd.masks, pd.b)
    r = np.random.default_rng(n + L)
    x = r.standard_normal(n) + 1j * r.standard_normal(n)
    w = r.standard_normal(L * n)
    yo = prob.C_apply(x) + prob.Astar_apply(w, x)
    hp = S.scgal_create_phase(pd.masks, L, n, pd.b, 0.0,
                              S.scgal_params_default(R=3, T_max=10, precision=prec, fft=S.SCGAL_FFT_PASSES))
    assert S.scgal_get_info(hp)["fft_cluster"] == 0
    yp = S.scgal_apply_D(hp, x, w)
    if not fits:
        with pytest.raises(S.ScgalError):
            S.scgal_create_phase(pd.masks, L, n, pd.b, 0.0,
                                 S.scgal_params_default(R=3, T_max=10, precision=prec, fft=S.SCGAL_FFT_CLUSTER))
        assert S.scgal_get_info(S.scgal_create_phase(
            pd.masks, L, n, pd.b, 0.0, S.scgal_params_default(R=3, T_max=10, precision=prec)))["fft_cluster"] == 0
        return
    hc = S.scgal_create_phase(pd.masks, L, n, pd.b, 0.0,
                              S.scgal_params_default(R=3, T_max=10, precision=prec, fft=S.SCGAL_FFT_CLUSTER))
    assert S.scgal_get_info(hc)["fft_cluster"] == C
    ha = S.scgal_create_phase(pd.masks, L, n, pd.b, 0.0, S.scgal_params_default(R=3, T_max=10, precision=prec))
    # AUTO: the clustered kernel for FP32 wherever it fits, for FP64 with 16-block clusters
    assert S.scgal_get_info(ha)["fft_cluster"] == (C if prec == 32 or C == 16 else 0)
    yc = S.scgal_apply_D(hc, x, w)
    assert _relerr(yc, yo) <= TOL_MV[prec]
    assert np.max(np.abs(yc - yo)) <= TOL_MV[prec] * np.max(np.abs(yo))
    assert _relerr(yc, yp) <= 2 * TOL_MV[prec]
    np.testing.assert_array_equal(S.scgal_apply_D(hc, x, w), yc)   # deterministic


def test_cluster_kernel_rejects_small_transforms(S):
    pd = W.phase_problem(128, 2, seed=0)   # n2 = 8 < 16 points
    with pytest.raises(S.ScgalError):
        S.scgal_create_phase(pd.masks, 2, 128, pd.b, 0.0, S.scgal_params_default(T_max=5, fft=S.SCGAL_FFT_CLUSTER))
    h = S.scgal_create_phase(pd.masks, 2, 128, pd.b, 0.0, S.scgal_params_default(T_max=5))
    assert S.scgal_get_info(h)["fft_cluster"] == 0


@pytest.mark.parametrize("prec", [32, 64])
def test_cluster_and_passes_solves_agree(S, prec):
    """Thirty iterations of Alg. 6.1 on the n = 2^12 coded-diffraction problem with
    each D-matvec kernel (the Lanczos steps and the primal update both change):
    the records agree to rounding, and each path repeats itself bitwise."""
    n, L, T = 4096, 12, 30
    recs = {}
    for fft in (S.SCGAL_FFT_PASSES, S.SCGAL_FFT_CLUSTER):
        runs = []
        for _ in range(2):
            pd, h, prob = _pair(S, n, L, prec, R=5, T_max=T, fft=fft)
            S.scgal_solve(h, T)
            runs.append((S.scgal_history(h, 1, T), S.scgal_get_state(h)["z"]))
        for a, b in zip(runs[0][0], runs[1][0]):
            assert a == b
        np.testing.assert_array_equal(runs[0][1], runs[1][1])
        recs[fft] = runs[0]
    tol = TOL_E2E[prec]
    for a, b in zip(recs[S.SCGAL_FFT_PASSES][0], recs[S.SCGAL_FFT_CLUSTER][0]):
        assert abs(a["xi"] - b["xi"]) <= tol * abs(a["xi"])
        assert abs(a["p"] - b["p"]) <= tol * abs(a["p"])
        assert abs(a["infeas"] - b["infeas"]) <= tol * a["infeas"]
    zp, zc = recs[S.SCGAL_FFT_PASSES][1], recs[S.SCGAL_FFT_CLUSTER][1]
    assert np.linalg.norm(zp - zc) <= tol * np.linalg.norm(zp)


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
