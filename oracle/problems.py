"""Problem data behind the three black-box primitives of Eq. 2.3 (oracle side).

A problem instance is the tuple (C, A, b, alpha) of Eq. 2.2.  SketchyCGAL only
touches it through
    (1) u -> C u,   (2) (u, z) -> (A* z) u,   (3) u -> A(u u*).
Both classes below expose these primitives for the *scaled* instance of
Eq. 7.1 (||C||_F = ||A|| = alpha = 1, all ||A_i||_F equal) when ``scale`` is
true, together with the factors that map scaled quantities back to the
original data (metrics are reported on the original data, Section 7.2.5).

Scaling (Eq. 7.1).  With X = alpha X', the instance becomes
    min <C', X'>  s.t.  A' X' = b',  X' in Delta_n
    C' = C / ||C||_F,   A' = A / ||A||,   b' = b / (alpha ||A||),
and  <C, X> = alpha ||C||_F <C', X'>,  A X - b = alpha ||A|| (A' X' - b').
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


class MaxCutProblem:
    """MaxCut SDP of Eq. 1.2 as an instance of Eq. 2.2.

    Laplacian L = sum_{ij in E} w_ij (e_i - e_j)(e_i - e_j)^T (Eq. 1.1 with edge
    weights), C = -L/4, A = diag (A_i = e_i e_i^T, so ||A|| = 1), b = 1,
    alpha = n.  Primitives (Section 2.4):
        (1) u -> -L u / 4,  (2) (u, z) -> z .* u,  (3) u -> |u|^2.
    The SDP optimum of Eq. 1.2 (maximise tr(L X)/4) equals -p*.
    """

    complex_ = False

    def __init__(self, n: int, ei, ej, w, scale: bool = True, alpha: float | None = None):
        self.n = int(n)
        self.d = self.n
        ei = np.asarray(ei, dtype=np.int64)
        ej = np.asarray(ej, dtype=np.int64)
        w = np.asarray(w, dtype=np.float64)
        W = sp.coo_matrix((np.concatenate([w, w]), (np.concatenate([ei, ej]), np.concatenate([ej, ei]))),
                          shape=(n, n)).tocsr()
        self.deg = np.asarray(W.sum(axis=1)).ravel()
        self.L = (sp.diags(self.deg) - W).tocsr()
        self.edges = (ei, ej, w)
        # ||C||_F = ||L||_F / 4 ; ||L||_F^2 = sum deg_i^2 + sum_{i != j} w_ij^2
        self.normC = 0.25 * math.sqrt(float(np.sum(self.deg ** 2) + 2.0 * np.sum(w ** 2)))
        self.normA = 1.0
        self.alpha_orig = float(n if alpha is None else alpha)
        self.b_orig = np.ones(self.n)
        self._set_scale(scale)

    def _set_scale(self, scale: bool):
        self.scaled = bool(scale)
        if scale:
            # Eq. 7.1 divides C by ||C||_F; when C = 0 (a graph without edges)
            # there is nothing to normalise and C' = C.
            cnorm = self.normC if self.normC > 0.0 else 1.0
            self.sC = 1.0 / cnorm
            self.sA = 1.0 / self.normA
            self.alpha = 1.0
            self.b = self.b_orig / (self.alpha_orig * self.normA)
            self.obj_factor = self.alpha_orig * cnorm        # <C,X> = obj_factor * <C',X'>
            self.z_factor = self.alpha_orig * self.normA     # AX - b = z_factor * (A'X' - b')
            self.X_factor = self.alpha_orig                  # X = X_factor * X'
            self.normA_s = 1.0
        else:
            self.sC = self.sA = 1.0
            self.alpha = self.alpha_orig
            self.b = self.b_orig.copy()
            self.obj_factor = self.z_factor = self.X_factor = 1.0
            self.normA_s = self.normA

    # primitive (1): u -> C u
    def C_apply(self, u):
        return self.sC * (-0.25) * (self.L @ u)

    # primitive (2): (u, z) -> (A* z) u
    def Astar_apply(self, z, u):
        return self.sA * z * u

    # primitive (3): u -> A(u u*)
    def A_of_uu(self, u):
        return self.sA * np.abs(u) ** 2

    def dense_C(self):
        return self.sC * (-0.25) * self.L.toarray()


class PhaseProblem:
    """Abstract phase retrieval SDP (Eq. 7.3) with coded diffraction patterns.

    Measurement vectors a_{(j-1)n+l} = W_n(l, :) diag(psi_j) (App. F.1), so
    <A_i, X> = |FFT(psi_j .* x)_l|^2 for X = x x*.  W is the unnormalised DFT,
    W(l, k) = exp(-2 pi i l k / n), and W* = n * ifft.  Then
        (1) u -> u                       (C = I)
        (2) (u, z) -> sum_j conj(psi_j) .* W*(z_j .* W(psi_j .* u))
        (3) u -> [ |W(psi_j .* u)|^2 ]_j        (mask-major, index j*n + l)
    With unit-modulus masks the Gram matrix G_ik = |a_i* a_k|^2 is entrywise
    nonnegative with every row summing to L n^2 (Parseval), so
    ||A|| = sqrt(lambda_max(G)) = n sqrt(L); ||C||_F = ||I||_F = sqrt(n).
    The problem is posed with tr X <= alpha (App. D.2 item 1), alpha = 3n.
    """

    complex_ = True

    def __init__(self, masks, b, alpha: float | None = None, scale: bool = True):
        self.masks = np.asarray(masks, dtype=np.complex128)
        self.L_masks, self.n = self.masks.shape
        self.d = self.L_masks * self.n
        self.b_orig = np.asarray(b, dtype=np.float64).reshape(-1)
        self.normA = self.n * math.sqrt(self.L_masks)
        self.normC = math.sqrt(self.n)
        self.alpha_orig = float(3 * self.n if alpha is None else alpha)
        self._set_scale(scale)

    _set_scale = MaxCutProblem._set_scale

    def C_apply(self, u):
        return self.sC * u

    def Astar_apply(self, z, u):
        Z = np.asarray(z).reshape(self.L_masks, self.n)
        F = np.fft.fft(self.masks * u[None, :], axis=1)
        back = self.n * np.fft.ifft(Z * F, axis=1)
        return self.sA * np.sum(np.conj(self.masks) * back, axis=0)

    def A_of_uu(self, u):
        F = np.fft.fft(self.masks * u[None, :], axis=1)
        return self.sA * (np.abs(F) ** 2).reshape(-1)

    def dense_C(self):
        return self.sC * np.eye(self.n, dtype=np.complex128)


def window_overlaps(N: int, M: int, s: int) -> np.ndarray:
    """ov[k] = |[0, M) intersect ([k s, k s + M) mod N)|, k = 0 .. N/s - 1 (one dimension)."""
    K = N // s
    base = np.zeros(N, dtype=bool)
    base[:M] = True
    ov = np.empty(K, dtype=np.int64)
    for k in range(K):
        w = np.zeros(N, dtype=bool)
        w[(k * s + np.arange(M)) % N] = True
        ov[k] = int(np.sum(base & w))
    return ov


class PtychoProblem:
    """Fourier-ptychography phase retrieval SDP (Section 7.4, App. F.2), same
    SDP as Eq. 7.3 (C = I, tr X <= alpha) with the measurement vectors
        a_{(j-1)m + l} = W*_m(l, :) Phi_j,
    where chi in C^n, n = N^2, is the Fourier-domain image (row-major N x N),
    Phi_j (m x n, one nonzero per row) selects the M x M aperture window of
    illumination j = (kr, kc), 0 <= kr, kc < K, at offset (kr s, kc s) with
    indices taken mod N, weighted by the pupil p (M x M, unit modulus):
        (Phi_j u)[r M + c] = p[r M + c] u[((kr s + r) mod N) N + (kc s + c) mod N],
    and W_m is the two-dimensional M x M DFT (m = M^2, unnormalised, row-major
    low-resolution pixel order), W*_m its conjugate transpose (= m ifft2).
    Primitives:
        (1) u -> u
        (2) (u, z) -> sum_j Phi_j^* W_m (z_j .* W*_m Phi_j u)
        (3) u -> [ |W*_m Phi_j u|^2 ]_j
    ||A||: with g_i = Phi_j^* W_m e_l (A_i = g_i g_i^*; |entries| = 1 on window j),
    sum over l' of |g_{j'l'}^* g_i|^2 = ||W*_m Phi_j' g_i||^2 = m |W_j cap W_j'|.
    On a regular periodic grid (K s = N) every row of the nonnegative Gram matrix
    G_ik = |g_i^* g_k|^2 has the sum m (sum_k ov(k))^2, so ||A||^2 = lambda_max(G)
    equals it (Perron-Frobenius): ||A|| = M sum_k ov(k).  ||C||_F = sqrt(n).
    alpha defaults to 1.5 for a unit-norm signal (Section 7.4.2).
    """

    complex_ = True

    def __init__(self, N: int, M: int, s: int, pupil, b, alpha: float | None = None, scale: bool = True):
        if N % s or M > N:
            raise ValueError("windows need s | N and M <= N")
        self.N, self.M, self.s, self.K = int(N), int(M), int(s), int(N // s)
        self.n = self.N * self.N
        self.m = self.M * self.M
        self.L_masks = self.K * self.K
        self.d = self.L_masks * self.m
        self.pupil = np.asarray(pupil, dtype=np.complex128).reshape(self.M, self.M)
        self.b_orig = np.asarray(b, dtype=np.float64).reshape(-1)
        self.normA = float(self.M * np.sum(window_overlaps(self.N, self.M, self.s)))
        self.normC = math.sqrt(self.n)
        self.alpha_orig = float(1.5 if alpha is None else alpha)
        r = np.arange(self.M)
        # pixel indices of every window: idx[j] is M x M
        self.idx = np.empty((self.L_masks, self.M, self.M), dtype=np.int64)
        for kr in range(self.K):
            for kc in range(self.K):
                rows = (kr * self.s + r) % self.N
                cols = (kc * self.s + r) % self.N
                self.idx[kr * self.K + kc] = rows[:, None] * self.N + cols[None, :]
        self._set_scale(scale)

    _set_scale = MaxCutProblem._set_scale

    def _forward(self, u):
        """W*_m Phi_j u for every j: L x M x M."""
        U = self.pupil[None, :, :] * np.asarray(u)[self.idx]
        return self.m * np.fft.ifft2(U, axes=(1, 2))

    def C_apply(self, u):
        return self.sC * u

    def Astar_apply(self, z, u):
        Z = np.asarray(z).reshape(self.L_masks, self.M, self.M)
        back = np.fft.fft2(Z * self._forward(u), axes=(1, 2))
        out = np.zeros(self.n, dtype=np.complex128)
        np.add.at(out, self.idx.reshape(-1), (np.conj(self.pupil)[None, :, :] * back).reshape(-1))
        return self.sA * out

    def A_of_uu(self, u):
        return self.sA * (np.abs(self._forward(u)) ** 2).reshape(-1)

    def dense_C(self):
        return self.sC * np.eye(self.n, dtype=np.complex128)
