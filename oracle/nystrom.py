"""NystromSketch (Alg. 5.1 with the trace and error additions of Alg. B.1), oracle side.

Sketch of a psd X: S = X Omega (Eq. 5.1) and tau = tr X (Eq. B.1), kept
under rank-one updates X <- (1-eta) X + eta v v* (Eq. 5.2 / Eq. B.2).

Reconstruct follows Alg. B.1 in its printed order:
    sigma   = sqrt(n) * eps(norm(S))          shift
    S_sigma = S + sigma * Omega               sketch of X + sigma I
    L       = chol(Omega* S_sigma)            upper triangular, L* L = Omega* S_sigma
    [U, Sigma, ~] = svd(S_sigma / L)          S_sigma L^{-1}, thin SVD
    Lambda  = max(0, Sigma^2 - sigma I)
    err     = tau - cumsum(diag Lambda)       Schatten-1 errors, Eq. B.4
Readings: ``norm`` is the spectral norm; ``eps(x)`` is the FP64 spacing at |x|,
2^(floor(log2 x) - 52); Omega* S_sigma is symmetrised before the Cholesky
factorisation; if the factorisation fails the shift is multiplied by 10 and
the factorisation retried, at most ``MAX_SHIFT_RETRIES`` times.  The ladder is
what lets a sketch whose entries carry FP32 rounding noise (the mixed-precision
path) factor with a shift just above that noise instead of one fixed to the
storage format.  Trace correction (Alg. 6.1 last line, App. B.4) adds
(alpha - tr Lambda)/R to every eigenvalue.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_triangular

MAX_SHIFT_RETRIES = 16


def eps_at(x: float, mantissa_bits: int = 52) -> float:
    """Spacing of the binary format with `mantissa_bits` fraction bits at |x|."""
    if x == 0.0:
        return 2.0 ** (-1022 if mantissa_bits == 52 else -126)
    return 2.0 ** (math.floor(math.log2(abs(x))) - mantissa_bits)


class NystromSketch:
    def __init__(self, Omega: np.ndarray):
        self.Omega = np.array(Omega)
        self.n, self.R = self.Omega.shape
        self.S = np.zeros_like(self.Omega)
        self.tau = 0.0

    def rank_one_update(self, v: np.ndarray, eta: float):
        """S <- (1-eta) S + eta v (v* Omega); tau <- (1-eta) tau + eta ||v||^2 (Eq. B.2)."""
        r = np.conj(v) @ self.Omega
        self.S = (1.0 - eta) * self.S + eta * np.outer(v, r)
        self.tau = (1.0 - eta) * self.tau + eta * float(np.real(np.vdot(v, v)))

    def scale(self, factor: float):
        """X <- factor X (the H = 0 branch of the trace-bounded LMO)."""
        self.S = factor * self.S
        self.tau = factor * self.tau

    def reconstruct(self):
        """Alg. B.1 Reconstruct: returns (U, Lambda (descending), err)."""
        n = self.n
        normS = float(np.linalg.norm(self.S, 2))
        sigma = math.sqrt(n) * eps_at(normS)
        self.shift_retries = 0
        for attempt in range(MAX_SHIFT_RETRIES + 1):
            self.shift_retries = attempt
            S_sig = self.S + sigma * self.Omega
            B = np.conj(self.Omega.T) @ S_sig
            B = 0.5 * (B + np.conj(B.T))
            try:
                G = np.linalg.cholesky(B)      # lower, G G* = B
            except np.linalg.LinAlgError:
                sigma *= 10.0
                continue
            Lup = np.conj(G.T)                 # upper, Lup* Lup = B
            # Y = S_sig Lup^{-1}  <=>  Lup^T Y^T = S_sig^T
            Y = solve_triangular(Lup, S_sig.T, trans="T", lower=False).T
            U, Sig, _ = np.linalg.svd(Y, full_matrices=False)
            Lam = np.maximum(0.0, Sig ** 2 - sigma)
            err = self.tau - np.cumsum(Lam)
            return U, Lam, err
        raise np.linalg.LinAlgError("Cholesky failed after every shift increase")


def trace_correct(Lam: np.ndarray, alpha: float) -> np.ndarray:
    """Lambda + (alpha - tr Lambda) I / R  (Alg. 6.1 optional step, Eq. B.5)."""
    return Lam + (alpha - float(np.sum(Lam))) / Lam.size
