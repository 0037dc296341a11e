"""Rounding and evaluation (oracle side).

* MaxCut (Section 7.2.1): the columns of sgn(U) are R cuts; evaluate each and
  keep the heaviest.  Readings: sgn(0) = +1; the weight of cut chi is
  sum_{ij in E} w_ij (1 - chi_i chi_j) / 2, accumulated in int64 when all
  weights are integers; ties go to the lowest column.
* Brute-force max cut for n <= 20 (test pin only).
* Phase retrieval (Section 7.3.2): chi = sqrt(lambda_1) u_1; relative error
  min_phi ||e^{i phi} chi - chi_true|| / ||chi_true|| (Section 7.3.3).
"""
from __future__ import annotations

import numpy as np


def sgn(x):
    return np.where(np.asarray(x) >= 0, 1, -1).astype(np.int64)


def cut_weight(ei, ej, w, chi):
    chi = np.asarray(chi)
    cut = chi[ei] != chi[ej]
    w = np.asarray(w)
    if np.all(w == np.round(w)):
        return int(np.sum(w[cut].astype(np.int64)))
    return float(np.sum(w[cut]))


def round_maxcut(U, ei, ej, w):
    cuts = [cut_weight(ei, ej, w, sgn(np.real(U[:, c]))) for c in range(U.shape[1])]
    best = int(np.argmax(cuts))  # argmax returns the first maximum
    return cuts[best], best, cuts


def brute_force_maxcut(n, ei, ej, w):
    if n > 22:
        raise ValueError("brute force limited to n <= 22")
    best = -np.inf
    ei = np.asarray(ei)
    ej = np.asarray(ej)
    w = np.asarray(w, dtype=np.float64)
    for chunk in range(0, 1 << (n - 1), 1 << 16):
        codes = np.arange(chunk, min(chunk + (1 << 16), 1 << (n - 1)), dtype=np.int64)
        bits = ((codes[:, None] >> np.arange(n - 1)[None, :]) & 1).astype(np.int8)
        side = np.concatenate([np.zeros((codes.size, 1), np.int8), bits], axis=1)  # vertex 0 fixed
        val = ((side[:, ei] != side[:, ej]) * w[None, :]).sum(axis=1)
        best = max(best, float(val.max()))
    return best


def phase_round(U, Lam):
    k = int(np.argmax(Lam))
    return np.sqrt(max(float(Lam[k]), 0.0)) * U[:, k]


def phase_error(chi, chi_true):
    c = np.vdot(chi, chi_true)
    ph = c / abs(c) if abs(c) > 0 else 1.0
    return float(np.linalg.norm(ph * chi - chi_true) / np.linalg.norm(chi_true))
