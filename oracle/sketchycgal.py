"""SketchyCGAL (Alg. 6.1), oracle side, FP64.

One iteration t = 1, 2, ... (Section 6.1):
    beta = beta0 sqrt(t+1),  eta = 2 / (t+1)
    (xi, v) = ApproxMinEvec(C + A*(y + beta (z - b)); q_t)          Eq. 6.1, Alg. 4.1
    z <- (1-eta) z + eta A(alpha v v*)                              Eq. 6.2, primitive (3)
    y <- y + gamma (z - b)                                          Eq. 6.3
        gamma = largest value with gamma ||z-b||^2 <= 4 alpha^2 beta0 ||A||^2 / (t+1)^{3/2}
                and 0 <= gamma <= beta0;  gamma = 0 if ||y_new|| > K  (Eq. 6.4)
    S <- (1-eta) S + eta alpha v (v* Omega)  (RankOneUpdate(sqrt(alpha) v, eta))
    p <- (1-eta) p + eta alpha v*(C v)                              Section 6.2.2
starting from z = y = 0, S = 0, p = 0, tau = 0; afterwards Reconstruct and the
optional trace correction.

Readings (where the paper is silent or ambiguous):
* v returned by ApproxMinEvec is renormalised to unit length; xi is the Ritz
  value lambda_min(T).
* The surrogate gap drops alpha in the printed formula; the maximum of
  <D, X - H> over H in alpha Delta is <D, X> - alpha lambda_min(D), so the
  stopping rule (Eq. E.1) uses alpha * xi (alpha * min(0, xi) for tr X <= alpha).
  Its numerator equals the bound of Eq. 6.6:
      p + <y, b> + beta/2 <z - b, z + b> - alpha xi.
  lambda_min(D_t) is replaced by the inexact xi_t of the same iteration (App. E).
  The rule is evaluated on the state of iteration t before its update, in the
  original units: relgap = obj_factor * num / (1 + obj_factor |p|),
  infeas = z_factor ||z - b|| / (1 + ||b_orig||).  On success the returned
  state is X_t (the update of iteration t is not applied).
* Trace-bounded LMO (App. D.2 item 1): if xi >= 0 the direction is H = 0, so
  z, S, tau, p are all scaled by (1 - eta).
* gamma = beta0 when z = b exactly.

General template (App. D, Alg. D.1) with the inclusion A(X) in K instead of
A(X) = b, for K = {b} ("eq", the model problem) or K = {u : u <= b} ("leq",
inequality constraints, App. D.3 item 1), through the slack w in K:
    w = proj_K(z + y / beta)                       gradient weights y + beta (z - w)
    wbar = proj_K(z_new + y / beta_+), beta_+ = beta0 sqrt(t+2)
    y <- y + gamma (z_new - wbar),  gamma ||z_new - wbar||^2 <= beta eta^2 alpha^2 ||A||^2
(the last bound equals the one of Eq. 6.4).  Readings:
* proj onto {u <= b} is the componentwise min(w, b), i.e. b + (w - b)_-; the
  paper prints (w - b)_-, which is that projection less b.
* The paper states no stopping rule for the template.  The bound of Eq. 6.6
  repeated with the slack (convexity of the augmented Lagrangian in X, and
  L(X*) <= p* at w = A X* for a feasible X*) gives
      p - p* <= p + <y, w> + beta/2 <z - w, z + w> - alpha xi,
  which is Eq. E.1's numerator with b replaced by w = proj_K(z + y / beta);
  the infeasibility is the distance to K, ||z - proj_K(z)|| / (1 + ||b||).
  For K = {b} both are exactly Eq. E.1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .lanczos import approx_min_evec, lanczos_steps
from .nystrom import NystromSketch, trace_correct as _trace_correct
from .philox import PURPOSE_LANCZOS, PURPOSE_OMEGA, gaussian_matrix, gaussian_vector


@dataclass
class SolveResult:
    U: np.ndarray
    Lam: np.ndarray           # eigenvalues of the reconstruction, original scale
    err: np.ndarray           # Schatten-1 errors, original scale
    z: np.ndarray             # scaled state
    y: np.ndarray
    p: float
    tau: float
    S: np.ndarray
    Omega: np.ndarray
    t_done: int               # iterations whose update was applied
    converged_at: int | None
    history: list = field(default_factory=list)
    vs: list | None = None    # unit vectors v_t (if recorded)


def dual_step(normsq_zb: float, t: int, alpha: float, beta0: float, normA: float) -> float:
    """Largest gamma in [0, beta0] with gamma ||z-b||^2 <= 4 alpha^2 beta0 ||A||^2 / (t+1)^{3/2} (Eq. 6.4)."""
    if normsq_zb == 0.0:
        return beta0
    return min(beta0, 4.0 * alpha * alpha * beta0 * normA * normA / ((t + 1) ** 1.5 * normsq_zb))


def proj_K(u, b, kset: str):
    """Euclidean projection onto K (App. D.3): K = {b}, or K = {u <= b}."""
    if kset == "eq":
        return b
    if kset == "leq":
        return np.minimum(u, b)
    raise ValueError(kset)


def al_weights(z, y, beta, b, kset: str):
    """Weights u = y + beta (z - w) of D = C + A*(u) (Alg. D.1), with the slack
    w = proj_K(z + y / beta); for K = {b}, w = b (Eq. 6.1)."""
    if kset == "eq":
        return y + beta * (z - b)
    return y + beta * (z - proj_K(z + y / beta, b, kset))


def stopping_values(prob, p, y, z, beta, xi, lmo, kset: str = "eq"):
    """Relative gap and infeasibility of Eq. E.1 in the original units (for
    K = {u <= b}: b replaced by the slack w = proj_K(z + y / beta) in the gap,
    and the infeasibility measured as the distance of z to K)."""
    b = prob.b
    w = b if kset == "eq" else proj_K(z + y / beta, b, kset)
    lam_term = prob.alpha * (min(0.0, xi) if lmo == "leq" else xi)
    num = p + float(np.dot(y, w)) + 0.5 * beta * float(np.dot(z - w, z + w)) - lam_term
    p_orig = prob.obj_factor * p
    relgap = prob.obj_factor * num / (1.0 + abs(p_orig))
    dz = z - proj_K(z, b, kset)
    infeas = prob.z_factor * float(np.linalg.norm(dz)) / (1.0 + float(np.linalg.norm(prob.b_orig)))
    return relgap, infeas, p_orig


def sketchy_cgal(prob, R: int, T: int, seed: int = 0, instance: int = 0, beta0: float = 1.0,
                 K: float = math.inf, lmo: str | None = None, trace_correct: bool | None = None,
                 tol: float | None = None, store_basis: bool = True,
                 record_v: bool = False, t_start: int = 1, kset: str = "eq") -> SolveResult:
    """Run Alg. 6.1 for t = t_start .. T (t_start > 1 only for timing samples);
    kset = "leq" runs Alg. D.1 with K = {u : u <= b}."""
    n, d = prob.n, prob.d
    cplx = prob.complex_
    if lmo is None:
        lmo = "leq" if cplx else "eq"
    if trace_correct is None:
        trace_correct = (lmo == "eq")
    alpha = prob.alpha
    Omega = gaussian_matrix(seed, PURPOSE_OMEGA, instance, n, R, cplx)
    sketch = NystromSketch(Omega)
    z = np.zeros(d)
    y = np.zeros(d)
    p = 0.0
    hist = []
    vs = [] if record_v else None
    converged_at = None
    t_done = 0
    for t in range(t_start, T + 1):
        beta = beta0 * math.sqrt(t + 1)
        eta = 2.0 / (t + 1)
        w = al_weights(z, y, beta, prob.b, kset)

        def Mv(u, w=w):
            return prob.C_apply(u) + prob.Astar_apply(w, u)

        q = lanczos_steps(n, t)
        v1 = gaussian_vector(seed, PURPOSE_LANCZOS, t, instance, n, cplx)
        xi, v, info = approx_min_evec(Mv, v1, q, store_basis)
        v = v / np.linalg.norm(v)
        relgap, infeas, p_orig = stopping_values(prob, p, y, z, beta, xi, lmo, kset)
        rec = dict(t=t, q=q, k=info["k"], xi=xi, p=p, p_orig=p_orig, relgap=relgap, infeas=infeas)
        if tol is not None and relgap <= tol and infeas <= tol:
            rec["gamma"] = 0.0
            hist.append(rec)
            converged_at = t
            break
        if lmo == "leq" and xi >= 0.0:
            z = (1.0 - eta) * z
            sketch.scale(1.0 - eta)
            p = (1.0 - eta) * p
            h_taken = False
        else:
            h = prob.A_of_uu(math.sqrt(alpha) * v)           # A(alpha v v*)
            z = (1.0 - eta) * z + eta * h
            vCv = float(np.real(np.vdot(v, prob.C_apply(v))))
            p = (1.0 - eta) * p + eta * alpha * vCv
            sketch.rank_one_update(math.sqrt(alpha) * v, eta)
            h_taken = True
        if kset == "eq":
            zb = z - prob.b
        else:
            zb = z - proj_K(z + y / (beta0 * math.sqrt(t + 2)), prob.b, kset)
        nzb2 = float(np.dot(zb, zb))
        gamma = dual_step(nzb2, t, alpha, beta0, prob.normA_s)
        y_new = y + gamma * zb
        if math.isfinite(K) and float(np.linalg.norm(y_new)) > K:
            gamma = 0.0
            y_new = y
        y = y_new
        rec["gamma"] = gamma
        rec["h"] = h_taken
        hist.append(rec)
        if record_v:
            vs.append(v.copy())
        t_done = t
    U, Lam, err = sketch.reconstruct()
    if trace_correct:
        Lam = _trace_correct(Lam, alpha)
    f = prob.X_factor
    return SolveResult(U=U, Lam=f * Lam, err=f * err, z=z, y=y, p=p, tau=sketch.tau, S=sketch.S,
                       Omega=Omega, t_done=t_done, converged_at=converged_at, history=hist, vs=vs)
