"""Pins for the oracle's NystromSketch (Alg. 5.1 / B.1) on dense psd inputs."""
import math

import numpy as np
import pytest

from oracle.nystrom import NystromSketch, eps_at, trace_correct


def _psd(n, rank, seed, complex_=False, decay=None):
    r = np.random.default_rng(seed)
    G = r.standard_normal((n, rank)) + (1j * r.standard_normal((n, rank)) if complex_ else 0)
    Q, _ = np.linalg.qr(G)
    ev = np.linspace(3.0, 1.0, rank) if decay is None else decay
    return (Q * ev) @ np.conj(Q.T)


def _omega(n, R, seed, complex_=False):
    r = np.random.default_rng(seed)
    O = r.standard_normal((n, R))
    if complex_:
        O = O + 1j * r.standard_normal((n, R))
    return O


def _sketch_of(X, Omega, updates=None):
    sk = NystromSketch(Omega)
    sk.S = X @ Omega
    sk.tau = float(np.real(np.trace(X)))
    return sk


@pytest.mark.parametrize("complex_", [False, True])
@pytest.mark.parametrize("rank,R", [(1, 5), (3, 5), (5, 5), (4, 10)])
def test_exact_for_rank_at_most_R(rank, R, complex_):
    """rank X = r <= R  =>  X_hat = X (App. B.5, 'with probability one')."""
    n = 120
    X = _psd(n, rank, 1, complex_)
    sk = _sketch_of(X, _omega(n, R, 2, complex_))
    U, Lam, err = sk.reconstruct()
    Xh = (U * Lam) @ np.conj(U.T)
    assert np.linalg.norm(X - Xh) / np.linalg.norm(X) <= 1e-10
    np.testing.assert_allclose(np.conj(U.T) @ U, np.eye(R), atol=1e-10)
    assert np.all(Lam >= 0) and np.all(np.diff(Lam) <= 1e-12)


def test_rank_one_updates_track_X():
    """S and tau follow X under X <- (1-eta) X + eta v v* (Eq. B.2)."""
    n, R = 60, 6
    r = np.random.default_rng(3)
    Omega = _omega(n, R, 4)
    sk = NystromSketch(Omega)
    X = np.zeros((n, n))
    for t in range(1, 30):
        v = r.standard_normal(n)
        eta = 2.0 / (t + 1)
        X = (1 - eta) * X + eta * np.outer(v, v)
        sk.rank_one_update(v, eta)
    np.testing.assert_allclose(sk.S, X @ Omega, rtol=1e-12, atol=1e-12)
    assert math.isclose(sk.tau, np.trace(X), rel_tol=1e-12)


def test_error_formula_is_schatten1_error():
    """err_r = tau - tr[[X_hat]]_r equals ||X - [[X_hat]]_r||_* (Eq. B.4), and
    bounds the best rank-r error of X from above (Eq. B.5)."""
    n, R = 80, 8
    ev = 2.0 ** -np.arange(20)
    X = _psd(n, 20, 5, decay=ev)
    sk = _sketch_of(X, _omega(n, R, 6))
    U, Lam, err = sk.reconstruct()
    lamX = np.sort(np.linalg.eigvalsh(X))[::-1]
    for r in range(1, R + 1):
        Xr = (U[:, :r] * Lam[:r]) @ U[:, :r].T
        true = np.sum(np.abs(np.linalg.eigvalsh(X - Xr)))
        assert math.isclose(err[r - 1], true, rel_tol=1e-8, abs_tol=1e-12)
        assert np.sum(lamX[r:]) <= err[r - 1] + 1e-12
    assert np.all(np.diff(err) <= 1e-14)  # monotone in r


def test_trace_correction():
    """tr X_tilde = alpha and ||X - X_tilde||_* <= 2 ||X - X_hat||_* (App. B.4)."""
    n, R = 70, 5
    X = _psd(n, 15, 7, decay=np.linspace(1, 0.01, 15))
    alpha = float(np.trace(X))
    sk = _sketch_of(X, _omega(n, R, 8))
    U, Lam, err = sk.reconstruct()
    Lt = trace_correct(Lam, alpha)
    assert math.isclose(np.sum(Lt), alpha, rel_tol=1e-12)
    Xh = (U * Lam) @ U.T
    Xt = (U * Lt) @ U.T
    nuc = lambda A: np.sum(np.abs(np.linalg.eigvalsh(A)))
    assert nuc(X - Xt) <= 2 * nuc(X - Xh) + 1e-12


def test_eps_at():
    assert eps_at(1.0) == np.spacing(1.0)
    assert eps_at(3.7) == np.spacing(3.7)
    assert eps_at(3.7, 23) == float(np.spacing(np.float32(3.7)))
    assert eps_at(1e-5, 23) == float(np.spacing(np.float32(1e-5)))


@pytest.mark.parametrize("n,rank", [(100, 1), (800, 2), (5000, 9)])
def test_fp32_noisy_sketch_reconstructs_via_shift_ladder(n, rank):
    """A sketch whose entries carry FP32-level rounding noise (the mixed-precision
    path) is indefinite at the FP64 shift; the x10 ladder climbs to a shift just
    above the noise and the rank-r part is recovered to FP32 accuracy."""
    R = 10
    X = _psd(n, rank, 9)
    r = np.random.default_rng(10)
    Omega = _omega(n, R, 11).astype(np.float32).astype(np.float64)
    sk = NystromSketch(Omega)
    S = (X @ Omega).astype(np.float32).astype(np.float64)
    sk.S = S * (1 + 1e-6 * r.standard_normal(S.shape))
    sk.tau = float(np.trace(X))
    U, Lam, err = sk.reconstruct()
    lamX = np.sort(np.linalg.eigvalsh(X))[::-1][:rank]
    np.testing.assert_allclose(Lam[:rank], lamX, rtol=1e-4)
    Xh = (U[:, :rank] * Lam[:rank]) @ U[:, :rank].T
    assert np.linalg.norm(X - Xh) / np.linalg.norm(X) <= 1e-4
