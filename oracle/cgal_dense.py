"""CGAL with an explicit matrix iterate (Alg. 3.1), for tiny n only (oracle side).

This is the method SketchyCGAL tracks implicitly (Section 6.2): with the same
directions v_t, the implicit iterate X_t satisfies the loop invariants of
Eq. 6.5 (z_t = A X_t, S_t = X_t Omega, and, from Section 6.2.2,
p_t = <C, X_t>, tau_t = tr X_t).  The instance is built here from explicit
dense matrices C and A_1..A_d taken straight from the definitions (Eq. 1.1,
Eq. 1.2, Eq. 7.2, App. F.1) and scaled numerically (Eq. 7.1): ||C||_F by the
Frobenius norm, ||A|| as the square root of the top eigenvalue of the Gram
matrix [<A_i, A_k>].  Nothing is shared with ``problems.py``.
"""
from __future__ import annotations

import math

import numpy as np


def dense_maxcut(n, ei, ej, w):
    """C = -L/4 with L = sum w_ij (e_i - e_j)(e_i - e_j)^T; A_i = e_i e_i^T; b = 1; alpha = n."""
    L = np.zeros((n, n))
    for i, j, wij in zip(ei, ej, w):
        e = np.zeros(n)
        e[i], e[j] = 1.0, -1.0
        L += wij * np.outer(e, e)
    C = -L / 4.0
    As = np.zeros((n, n, n))
    for i in range(n):
        As[i, i, i] = 1.0
    return C, As, np.ones(n), float(n)


def dense_phase(masks, b, alpha=None):
    """C = I; A_i = a_i a_i* with a_i* x = (DFT (psi_j .* x))_l; tr X <= alpha = 3n."""
    L, n = masks.shape
    k = np.arange(n)
    Wn = np.exp(-2j * np.pi * np.outer(k, k) / n)
    As = []
    for j in range(L):
        for l in range(n):
            row = Wn[l, :] * masks[j, :]          # a_i* as a row: a_i* x = row . x
            a = np.conj(row)
            As.append(np.outer(a, np.conj(a)))
    return np.eye(n, dtype=np.complex128), np.array(As), np.asarray(b, dtype=np.float64), \
        float(3 * n if alpha is None else alpha)


def operator_norm(As):
    """||A||_{F -> l2} = sqrt(lambda_max(G)), G_ik = <A_i, A_k> (real for Hermitian A_i)."""
    d = As.shape[0]
    flat = As.reshape(d, -1)
    G = np.real(np.conj(flat) @ flat.T)
    return math.sqrt(float(np.linalg.eigvalsh(0.5 * (G + G.T))[-1]))


def scale_dense(C, As, b, alpha):
    normC = float(np.linalg.norm(C, "fro"))
    normA = operator_norm(As)
    return dict(C=C / normC, As=As / normA, b=b / (alpha * normA), alpha=1.0,
                normC=normC, normA=normA, obj_factor=alpha * normC, z_factor=alpha * normA)


def A_map(As, X):
    return np.real(np.einsum("kij,ij->k", np.conj(As), X))


def Astar_map(As, z):
    return np.einsum("k,kij->ij", z, As)


def cgal_dense(C, As, b, alpha, T, vs=None, h_flags=None, beta0=1.0, Omega=None):
    """Alg. 3.1 from X = 0, y = 0.  If ``vs`` is given, v_t = vs[t-1] (and
    h_flags[t-1] False means H_t = 0); otherwise v_t is an exact minimum
    eigenvector of D_t from a dense eigensolver.  Returns per-iteration records
    of X_{t+1}, A X_{t+1}, X_{t+1} Omega, <C, X_{t+1}>, tr X_{t+1}, y_{t+1}."""
    n = C.shape[0]
    X = np.zeros((n, n), dtype=C.dtype)
    y = np.zeros(As.shape[0])
    normA = operator_norm(As)
    recs = []
    for t in range(1, T + 1):
        beta = beta0 * math.sqrt(t + 1)
        eta = 2.0 / (t + 1)
        D = C + Astar_map(As, y + beta * (A_map(As, X) - b))
        lam, V = np.linalg.eigh(0.5 * (D + np.conj(D.T)))
        if vs is None:
            v = V[:, 0]
            take = True
        else:
            v = vs[t - 1]
            take = True if h_flags is None else bool(h_flags[t - 1])
        H = alpha * np.outer(v, np.conj(v)) if take else np.zeros_like(X)
        X = (1.0 - eta) * X + eta * H
        r = A_map(As, X) - b
        nr2 = float(np.dot(r, r))
        gamma = beta0 if nr2 == 0.0 else min(beta0, 4 * alpha**2 * beta0 * normA**2 / ((t + 1) ** 1.5 * nr2))
        y = y + gamma * r
        rec = dict(t=t, X=X.copy(), z=A_map(As, X), p=float(np.real(np.trace(C @ X))),
                   tau=float(np.real(np.trace(X))), y=y.copy(), lam_min=float(lam[0]),
                   normD=float(np.max(np.abs(lam))), D=D)
        if Omega is not None:
            rec["S"] = X @ Omega
        recs.append(rec)
    return recs
