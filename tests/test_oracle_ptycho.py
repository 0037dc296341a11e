"""Pins for the oracle's Fourier-ptychography operator (Section 7.4, App. F.2).

* The FFT-based primitives against the definition written with explicit
  matrices: a_{(j-1)m+l} = W*_m(l, :) Phi_j, W_m the M x M two-dimensional DFT
  as the Kronecker product of 1-D DFT matrices, Phi_j built entry by entry
  from the window rule.
* ||A|| (closed form on a periodic window grid) against lambda_max of the
  explicit Gram matrix G_ik = |a_i^* a_k|^2, also with windows that overlap by
  a non-multiple of the step.
* The measurement identity b = A(chi chi*) on the synthetic data.
* End to end: noiseless measurements with 16 intensities per real unknown
  have the rank-one solution chi chi*; SketchyCGAL recovers chi (up to a global
  phase) to 2e-2 relative error (the paper's target is 1e-2, Section 7.3.3).
"""
import numpy as np
import pytest

import workloads as W
from oracle.problems import PtychoProblem, window_overlaps
from oracle.rounding import phase_error, phase_round
from oracle.sketchycgal import sketchy_cgal


def _explicit_rows(N, M, s, pupil):
    """[A_j] with A_j = W_m^H Phi_j (m x n), from the definition."""
    K = N // s
    m, n = M * M, N * N
    W1 = np.exp(-2j * np.pi * np.outer(np.arange(M), np.arange(M)) / M)
    Wm = np.kron(W1, W1)
    p = np.asarray(pupil).reshape(-1)
    out = []
    for kr in range(K):
        for kc in range(K):
            Phi = np.zeros((m, n), dtype=np.complex128)
            for r in range(M):
                for c in range(M):
                    Phi[r * M + c, ((kr * s + r) % N) * N + (kc * s + c) % N] = p[r * M + c]
            out.append(Wm.conj().T @ Phi)
    return out


@pytest.mark.parametrize("N,M,s", [(12, 4, 3), (12, 5, 3), (8, 4, 2)])
def test_primitives_match_explicit_matrices(N, M, s):
    r = np.random.default_rng(N + M + s)
    pupil = np.exp(2j * np.pi * r.random(M * M))
    prob = PtychoProblem(N, M, s, pupil, np.zeros((N // s) ** 2 * M * M), scale=False)
    A = _explicit_rows(N, M, s, pupil)
    u = r.standard_normal(N * N) + 1j * r.standard_normal(N * N)
    z = r.standard_normal(prob.d)
    meas = np.concatenate([np.abs(Aj @ u) ** 2 for Aj in A])
    np.testing.assert_allclose(prob.A_of_uu(u), meas, rtol=1e-11, atol=1e-9 * meas.max())
    Z = z.reshape(len(A), M * M)
    ref = sum(Aj.conj().T @ (Z[j] * (Aj @ u)) for j, Aj in enumerate(A))
    got = prob.Astar_apply(z, u)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)
    # adjoint identity u* (A* z) u = <z, A(u u*)>
    lhs = np.vdot(u, got).real
    assert abs(lhs - float(np.dot(z, meas))) <= 1e-10 * abs(lhs)


@pytest.mark.parametrize("N,M,s", [(12, 4, 3), (12, 5, 3), (8, 4, 2), (12, 6, 4)])
def test_operator_norm_closed_form(N, M, s):
    pupil = np.exp(2j * np.pi * np.random.default_rng(1).random(M * M))
    prob = PtychoProblem(N, M, s, pupil, np.zeros((N // s) ** 2 * M * M), scale=False)
    Afull = np.vstack(_explicit_rows(N, M, s, pupil))
    G = np.abs(Afull @ Afull.conj().T) ** 2
    lam = np.linalg.eigvalsh(G)[-1]
    assert abs(np.sqrt(lam) - prob.normA) <= 1e-9 * prob.normA
    assert prob.normA == M * window_overlaps(N, M, s).sum()


def test_measurements_are_A_of_chi():
    pd = W.ptycho_problem(16, 8, 2, seed=3)
    prob = PtychoProblem(16, 8, 2, pd.pupil, pd.b, scale=False)
    np.testing.assert_allclose(prob.A_of_uu(pd.chi), pd.b, rtol=1e-10, atol=1e-12 * pd.b.max())
    assert abs(np.linalg.norm(pd.chi) - 1.0) <= 1e-12
    assert np.allclose(np.abs(pd.pupil), 1.0)


def test_recovers_signal():
    pd = W.ptycho_problem(16, 8, 2, seed=0)
    prob = PtychoProblem(16, 8, 2, pd.pupil, pd.b)
    res = sketchy_cgal(prob, R=5, T=1500, seed=0)
    h = res.history[-1]
    assert h["relgap"] <= 2e-3 and h["infeas"] <= 5e-3
    assert phase_error(phase_round(res.U, res.Lam), pd.chi) < 2e-2
