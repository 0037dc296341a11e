"""ApproxMinEvec by randomized Lanczos (Alg. 4.1), oracle side.

Readings taken where the printed algorithm is ambiguous:
* The norm taken after the three-term recurrence is that of the new vector
  v_{i+1} (standard Lanczos; the next line divides v_{i+1} by it).
* The loop runs i = 1 .. min(q, n-1); breakdown is the exact test rho_i == 0,
  after which T is i x i.  The last iteration's rho and v_{i+1} are not needed.
* The tridiagonal minimum eigenpair uses a library routine (LAPACK via
  scipy.linalg.eigh_tridiagonal), which the paper allows ("or just use eig").
* v is the Ritz vector sum_j u_j v_j; the caller renormalises it.

Two storage modes: ``store_basis=False`` is the storage-optimal form of
Alg. 4.1 (the recurrence is run a second time to regenerate v_2..v_i and form
the sum); ``store_basis=True`` keeps the basis (Remark 4.2).  In exact
arithmetic and in this deterministic code both give identical results.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import eigh_tridiagonal


def lanczos_steps(n: int, t: int) -> int:
    """q_t = t^{1/4} log n (Section 4.2 / Alg. 6.1), read as ceil(t^{1/4} ln n),
    capped by Alg. 4.1 at n - 1."""
    return int(min(math.ceil(t ** 0.25 * math.log(n)), n - 1))


def _recurrence(Mv, v1, imax, keep):
    """Run the three-term recurrence; returns (omegas, rhos, basis or None)."""
    omegas, rhos = [], []
    basis = [v1] if keep else None
    v_prev = np.zeros_like(v1)
    rho_prev = 0.0
    vi = v1
    for i in range(1, imax + 1):
        y = Mv(vi)
        omega = float(np.real(np.vdot(vi, y)))
        w = y - omega * vi - rho_prev * v_prev
        omegas.append(omega)
        if i == imax:
            break
        rho = float(np.linalg.norm(w))
        if rho == 0.0:
            break
        w = w / rho
        rhos.append(rho)
        v_prev, vi, rho_prev = vi, w, rho
        if keep:
            basis.append(w)
    return omegas, rhos, basis


def tridiag_min_eig(omegas, rhos):
    """(xi, u): minimum eigenpair of tridiag(rho, omega, rho)."""
    d = np.asarray(omegas, dtype=np.float64)
    e = np.asarray(rhos[: len(d) - 1], dtype=np.float64)
    if d.size == 1:
        return float(d[0]), np.ones(1)
    w, U = eigh_tridiagonal(d, e, select="i", select_range=(0, 0))
    return float(w[0]), U[:, 0]


def approx_min_evec(Mv, v1, q: int, store_basis: bool = True):
    """Alg. 4.1.  Mv: u -> M u (Hermitian M); v1: the random start (unnormalised).

    Returns (xi, v, info) with xi = lambda_min(T) (the Ritz value), v the
    Ritz vector (not renormalised), info = dict(k, omegas, rhos).
    """
    n = v1.shape[0]
    v1 = v1 / np.linalg.norm(v1)
    imax = min(q, n - 1)
    omegas, rhos, basis = _recurrence(Mv, v1, imax, store_basis)
    k = len(omegas)
    xi, u = tridiag_min_eig(omegas, rhos)
    if store_basis:
        v = np.zeros_like(v1)
        for j in range(k):
            v = v + u[j] * basis[j]
    else:
        # regenerate v_1 .. v_k with the same recurrence and accumulate
        v = u[0] * v1
        v_prev = np.zeros_like(v1)
        vi = v1
        rho_prev = 0.0
        for j in range(1, k):
            y = Mv(vi)
            w = y - omegas[j - 1] * vi - rho_prev * v_prev
            w = w / rhos[j - 1]
            v_prev, vi, rho_prev = vi, w, rhos[j - 1]
            v = v + u[j] * vi
    return xi, v, dict(k=k, omegas=omegas, rhos=rhos[: k - 1])
