"""The storage-free test matrix (SCGAL_OMEGA_REGEN, Remark 5.2): Omega is never
stored and every use regenerates its rows from the counter-based stream.

Omega enters only the sketch (v* Omega in the Ritz step, and the
reconstruction), never the iterates z, y or the Lanczos runs, so the iteration
records of a regenerating solve equal the stored solve's bit for bit in both
precisions.  FP64 regeneration evaluates the same Box-Muller formula as the
stored draw, so the sketch and the reconstruction are bit-identical too; FP32
regeneration evaluates it in FP32 (within a few ulps of the rounded FP64 draw),
so the sketch agrees to 1e-5 relative and the reconstruction to 1e-4.
"""
import numpy as np
import pytest

import workloads as W
from oracle.nystrom import NystromSketch
from oracle.philox import PURPOSE_OMEGA, gaussian_matrix
from oracle.problems import MaxCutProblem
from oracle.sketchycgal import sketchy_cgal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_1912_02949_gb300 import build, scgal
    build.build()
    scgal.load()
    return scgal


def _mc(S, g, prec, omega, R=10, T_max=100, **kw):
    rp, col, val = g.csr()
    w = None if g.weight_kind == "unit" else val
    p = S.scgal_params_default(R=R, T_max=T_max, precision=prec, omega=omega, **kw)
    return S.scgal_create_maxcut(rp, col, w, g.n, col.size, 0.0, p)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("R", [10, 7])
def test_regenerated_omega_matches_stored(S, prec, R):
    """Odd R exercises rows that start in the middle of a normal pair."""
    g = W.er_graph(3000, 12000, seed=1, weights="pm1")
    T = 60
    a = _mc(S, g, prec, S.SCGAL_OMEGA_STORED, R=R, T_max=T)
    b = _mc(S, g, prec, S.SCGAL_OMEGA_REGEN, R=R, T_max=T)
    vb = 8 if prec == 64 else 4
    assert S.scgal_get_info(a)["device_bytes"] - S.scgal_get_info(b)["device_bytes"] == g.n * R * vb
    S.scgal_solve(a, T)
    S.scgal_solve(b, T)
    assert S.scgal_history(a, 1, T) == S.scgal_history(b, 1, T)
    sa, sb = S.scgal_get_state(a), S.scgal_get_state(b)
    assert sa["tau"] == sb["tau"] and sa["p"] == sb["p"]
    ra, rb = S.scgal_reconstruct(a), S.scgal_reconstruct(b)
    if prec == 64:
        assert np.array_equal(sa["S"], sb["S"])
        for x, y in zip(ra, rb):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    else:
        assert _rel(sb["S"], sa["S"]) <= 1e-5
        np.testing.assert_allclose(rb[1], ra[1], rtol=1e-4, atol=1e-4 * abs(ra[1][0]))
        assert abs(rb[3] - ra[3]) <= 1e-3 * abs(ra[3])


@pytest.mark.parametrize("prec", [32, 64])
def test_regenerated_omega_reconstructs_planted_sketch(S, prec):
    """Alg. B.1 on S = X Omega of a planted rank-3 psd X, Omega from the oracle's
    stream: the regenerating handle's reconstruction finds X's eigenvalues."""
    n, R = 3000, 8
    g = W.er_graph(n, 9000, seed=2, weights="unit")
    h = _mc(S, g, prec, S.SCGAL_OMEGA_REGEN, R=R, scale=0)
    Om = gaussian_matrix(0, PURPOSE_OMEGA, 0, n, R, False)
    r = np.random.default_rng(4)
    Q, _ = np.linalg.qr(r.standard_normal((n, 3)))
    ev = np.array([500.0, 200.0, 100.0])
    Sk = (Q * ev) @ (Q.T @ Om)
    tau = float(ev.sum())
    S.scgal_set_state(h, S=Sk, tau=tau, t=1)
    sk = NystromSketch(Om)
    sk.S = Sk
    sk.tau = tau
    Uo, Lo, eo = sk.reconstruct()
    U, lam, err, _ = S.scgal_reconstruct(h, want_cut=False)
    shift = (n - Lo.sum()) / R      # trace correction, on by default for MaxCut
    tol = 1e-4 if prec == 32 else 1e-8
    np.testing.assert_allclose(lam[:3] - shift, Lo[:3], rtol=tol)
    for c in range(3):
        assert abs(abs(np.dot(U[c], Uo[:, c])) - 1.0) <= tol


def test_regenerated_omega_small_basis(S):
    """T_max = 1 leaves a Lanczos basis smaller than n x R: the reconstruction
    regenerates Omega into a buffer of its own."""
    g = W.er_graph(100, 400, seed=3, weights="unit")
    a = _mc(S, g, 64, S.SCGAL_OMEGA_STORED, R=10, T_max=1)
    b = _mc(S, g, 64, S.SCGAL_OMEGA_REGEN, R=10, T_max=1)
    assert S.scgal_get_info(b)["qmax"] + 1 < 10
    S.scgal_solve(a, 1)
    S.scgal_solve(b, 1)
    ra, rb = S.scgal_reconstruct(a), S.scgal_reconstruct(b)
    for x, y in zip(ra, rb):
        assert np.array_equal(np.asarray(x), np.asarray(y))


def test_regenerated_omega_end_to_end_er800(S):
    """n = 800 Erdos-Renyi MaxCut, T = 500, FP32 with Omega regenerated: the
    objective within 1e-3 of the FP64 oracle, trace correction exact, and the
    reconstruction within 1e-4 of the stored-Omega solve (the FP32 trajectory
    itself follows the oracle only within its rounding spread; see
    test_gpu_maxcut)."""
    g = W.config_graph("er800")
    T = 500
    h = _mc(S, g, 32, S.SCGAL_OMEGA_REGEN, R=10, T_max=T)
    hs = _mc(S, g, 32, S.SCGAL_OMEGA_STORED, R=10, T_max=T)
    ref = sketchy_cgal(MaxCutProblem(g.n, g.i, g.j, g.w), R=10, T=T, seed=0)
    rc, last = S.scgal_solve(h, T)
    assert rc == S.SCGAL_ENOTDONE
    ro = ref.history[-1]
    assert abs(last["p"] - ro["p_orig"]) <= 1e-3 * abs(ro["p_orig"])
    U, lam, err, cut = S.scgal_reconstruct(h)
    assert abs(lam.sum() - ref.Lam.sum()) <= 1e-6 * ref.Lam.sum()
    S.scgal_solve(hs, T)
    _, lam_s, _, cut_s = S.scgal_reconstruct(hs)
    np.testing.assert_allclose(lam, lam_s, rtol=1e-4, atol=1e-4 * lam_s[0])
    assert abs(cut - cut_s) <= 1e-3 * cut_s


@pytest.mark.parametrize("prec", [32, 64])
def test_regenerated_omega_phase(S, prec):
    """Complex test matrix (phase retrieval): the same equalities."""
    n, L, T = 1024, 5, 40
    pd = W.phase_problem(n, L, seed=0)
    hs = [S.scgal_create_phase(pd.masks, L, n, pd.b, 0.0,
                               S.scgal_params_default(R=5, T_max=T, precision=prec, omega=om))
          for om in (S.SCGAL_OMEGA_STORED, S.SCGAL_OMEGA_REGEN)]
    vb = 16 if prec == 64 else 8
    assert S.scgal_get_info(hs[0])["device_bytes"] - S.scgal_get_info(hs[1])["device_bytes"] == n * 5 * vb
    for h in hs:
        S.scgal_solve(h, T)
    assert S.scgal_history(hs[0], 1, T) == S.scgal_history(hs[1], 1, T)
    ra, rb = S.scgal_reconstruct(hs[0], want_cut=False), S.scgal_reconstruct(hs[1], want_cut=False)
    if prec == 64:
        assert np.array_equal(ra[1], rb[1]) and np.array_equal(ra[0], rb[0])
    else:
        np.testing.assert_allclose(rb[1], ra[1], rtol=1e-4, atol=1e-4 * abs(ra[1][0]))


@pytest.mark.parametrize("n,deg", [(3000, 8), (20000, 6)])
def test_served_regenerated_omega(S, n, deg):
    """A served request that regenerates Omega runs on its own graphs (the
    batched kernels read a stored Omega): its objective equals a standalone
    stored-Omega solve's bit for bit, its cut and top eigenvalue agree to
    rounding."""
    g = W.er_graph(n, n * deg // 2, seed=11, weights="unit")
    rp, col, _ = g.csr()
    h = S.scgal_create_maxcut(rp, col, None, g.n, col.size, 0.0,
                              S.scgal_params_default(R=10, T_max=80, precision=32))
    rc, last = S.scgal_solve(h, 80)
    _, lam, _, cut = S.scgal_reconstruct(h)
    srv = S.scgal_server_create(1 << 32, 4)
    res = S.scgal_poll(srv, S.scgal_submit(srv, rp, col, None, g.n, col.size,
                                           S.scgal_params_default(R=10, T_max=80, precision=32,
                                                                  omega=S.SCGAL_OMEGA_REGEN)), -1)
    S.scgal_server_destroy(srv)
    assert res["status"] == S.SCGAL_ENOTDONE and res["iterations"] == 80
    assert res["objective"] == last["p"]
    assert abs(res["best_cut"] - cut) <= 1e-3 * cut
    assert abs(res["lambda_max"] - lam[0]) <= 1e-4 * lam[0]
