"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module only *generates problem data*: graphs (as edge lists and symmetric
CSR), phase-retrieval signals, masks and measurements, and request streams.  It
holds none of SketchyCGAL's arithmetic; both the FP64 oracle and the CUDA
library receive what it produces as plain arrays.

Shapes follow the workloads the paper evaluates (Section 7):

* MaxCut SDPs on sparse graphs (Gset / DIMACS10 shapes, Section 7.2) --
  Erdos-Renyi G(n, m), a 2-D torus with random long-range edges, and the
  log-uniform request mix used for serving.
* Abstract phase retrieval with coded diffraction patterns (Section 7.3,
  Appendix F.1): complex Gaussian signal, L modulating masks, and the
  intensity measurements |FFT(mask * x)|^2.

The paper's own datasets are not available; these generators stand in for
them (no item of those datasets is reproduced).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Graph", "er_graph", "torus_longrange_graph", "cycle_graph", "complete_graph",
    "csr_from_edges", "PhaseData", "phase_problem", "serving_requests",
    "config_graph",
]


@dataclass
class Graph:
    """Undirected weighted graph: edges (i[k], j[k]) with i < j, weight w[k]."""
    n: int
    i: np.ndarray  # int64[m]
    j: np.ndarray  # int64[m]
    w: np.ndarray  # float64[m]
    weight_kind: str  # "unit" | "pm1" | "real"

    @property
    def m(self) -> int:
        return int(self.i.shape[0])

    def csr(self):
        return csr_from_edges(self.n, self.i, self.j, self.w)


def _distinct_pairs(rng, n: int, m: int, exclude_keys=None) -> tuple[np.ndarray, np.ndarray]:
    """m distinct unordered pairs {i, j}, i != j, drawn uniformly (rejection)."""
    if m > n * (n - 1) // 2:
        raise ValueError("too many edges for a simple graph")
    keys = np.empty(0, dtype=np.int64)
    order = np.empty(0, dtype=np.int64)
    need = m
    pool_keys = []
    while need > 0:
        draw = int(need * 1.05) + 64
        a = rng.integers(0, n, size=draw, dtype=np.int64)
        b = rng.integers(0, n, size=draw, dtype=np.int64)
        ok = a != b
        a, b = a[ok], b[ok]
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        pool_keys.append(lo * n + hi)
        allk = np.concatenate(pool_keys)
        uk, first = np.unique(allk, return_index=True)
        if exclude_keys is not None and exclude_keys.size:
            keep = ~np.isin(uk, exclude_keys, assume_unique=False)
            uk, first = uk[keep], first[keep]
        # keep first occurrences in draw order so the subset is uniform
        sel = np.argsort(first, kind="stable")
        keys = uk[sel]
        order = first[sel]
        need = m - keys.size
    keys = keys[:m]
    return keys // n, keys % n


def er_graph(n: int, m: int, seed: int = 0, weights: str = "unit") -> Graph:
    """Erdos-Renyi G(n, m): m distinct uniform pairs, no self-loops.

    weights: "unit" (all 1) or "pm1" (+1/-1 with probability 1/2 each).
    """
    rng = np.random.default_rng(seed)
    i, j = _distinct_pairs(rng, n, m)
    w = _draw_weights(rng, m, weights)
    return Graph(n, i, j, w, weights)


def _draw_weights(rng, m: int, kind: str) -> np.ndarray:
    if kind == "unit":
        return np.ones(m, dtype=np.float64)
    if kind == "pm1":
        return (rng.integers(0, 2, size=m) * 2 - 1).astype(np.float64)
    if kind == "real":
        return rng.uniform(0.5, 1.5, size=m)
    raise ValueError(kind)


def torus_longrange_graph(rows: int, cols: int, extra_frac: float = 0.1, seed: int = 0,
                          weights: str = "pm1") -> Graph:
    """rows x cols 2-D torus (4-regular, 2n edges) plus extra_frac * 2n random
    long-range edges that duplicate no torus edge."""
    n = rows * cols
    r = np.arange(n, dtype=np.int64) // cols
    c = np.arange(n, dtype=np.int64) % cols
    right = r * cols + (c + 1) % cols
    down = ((r + 1) % rows) * cols + c
    src = np.concatenate([np.arange(n, dtype=np.int64)] * 2)
    dst = np.concatenate([right, down])
    lo, hi = np.minimum(src, dst), np.maximum(src, dst)
    tkeys = np.unique(lo * n + hi)
    rng = np.random.default_rng(seed)
    m_extra = int(round(extra_frac * tkeys.size))
    ei, ej = _distinct_pairs(rng, n, m_extra, exclude_keys=tkeys)
    i = np.concatenate([tkeys // n, ei])
    j = np.concatenate([tkeys % n, ej])
    w = _draw_weights(rng, i.size, weights)
    return Graph(n, i, j, w, weights)


def cycle_graph(n: int) -> Graph:
    i = np.arange(n, dtype=np.int64)
    j = (i + 1) % n
    lo, hi = np.minimum(i, j), np.maximum(i, j)
    return Graph(n, lo, hi, np.ones(n), "unit")


def complete_graph(n: int) -> Graph:
    i, j = np.triu_indices(n, 1)
    return Graph(n, i.astype(np.int64), j.astype(np.int64), np.ones(i.size), "unit")


def csr_from_edges(n: int, i: np.ndarray, j: np.ndarray, w: np.ndarray):
    """Symmetric CSR of the weighted adjacency (both directions, no diagonal).

    Returns (row_ptr int32[n+1], col int32[nnz], val float64[nnz]); columns are
    sorted within each row.
    """
    rows = np.concatenate([i, j]).astype(np.int64)
    cols = np.concatenate([j, i]).astype(np.int64)
    vals = np.concatenate([w, w]).astype(np.float64)
    key = rows * n + cols
    order = np.argsort(key, kind="stable")
    rows, cols, vals = rows[order], cols[order], vals[order]
    counts = np.bincount(rows, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz exceeds int32 CSR")
    return row_ptr.astype(np.int32), cols.astype(np.int32), vals


@dataclass
class PhaseData:
    """Coded-diffraction phase retrieval instance (Appendix F.1 shape)."""
    n: int
    L: int
    chi: np.ndarray    # complex128[n], the planted signal
    masks: np.ndarray  # complex128[L, n], entries in {1, -1, i, -i}
    b: np.ndarray      # float64[L * n], mask-major: b[j*n + l]


def phase_problem(n: int, L: int = 12, seed: int = 0) -> PhaseData:
    """chi ~ complex standard normal (real and imaginary parts N(0,1)); masks
    uniform on {1, -1, i, -i}; b = |FFT(mask_j * chi)|^2 (unnormalised DFT)."""
    rng = np.random.default_rng(seed)
    chi = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    phases = np.array([1, -1, 1j, -1j], dtype=np.complex128)
    masks = phases[rng.integers(0, 4, size=(L, n))]
    b = np.abs(np.fft.fft(masks * chi[None, :], axis=1)) ** 2
    return PhaseData(n, L, chi, masks, b.reshape(-1).astype(np.float64))


@dataclass
class PtychoData:
    N: int
    M: int
    s: int
    chi: np.ndarray      # Fourier-domain image, n = N^2, unit norm
    pupil: np.ndarray    # M x M, unit modulus
    b: np.ndarray        # L m intensities, window-major


def ptycho_problem(N: int = 320, M: int = 64, s: int = 20, seed: int = 0) -> PtychoData:
    """Synthetic Fourier-ptychography data in the shape of the paper's FP study
    (n = 320^2 image, 64^2-pixel low-resolution frames; App. F.2): a smooth
    nonnegative N x N image (a sum of 40 Gaussian blobs with random centres,
    widths N/40 .. N/8 and weights), chi = its unnormalised 2-D DFT scaled to
    unit norm; a K x K grid of periodic aperture windows (K = N / s) whose
    offsets overlap by M - s pixels; a unit-modulus defocus pupil
    exp(i pi (rho^2 / (M/2)^2) / 2); b = |W*_m Phi_j chi|^2 window by window."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:N, 0:N].astype(np.float64)
    img = np.zeros((N, N))
    for _ in range(40):
        cy, cx = rng.uniform(0, N, 2)
        w = rng.uniform(N / 40.0, N / 8.0)
        img += rng.uniform(0.2, 1.0) * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2 * w * w))
    chi = np.fft.fft2(img).reshape(-1)
    chi /= np.linalg.norm(chi)
    r = np.arange(M) - M / 2.0
    rho2 = r[:, None] ** 2 + r[None, :] ** 2
    pupil = np.exp(1j * np.pi * 0.5 * rho2 / (M / 2.0) ** 2)
    K = N // s
    out = np.empty((K * K, M, M))
    ar = np.arange(M)
    X = chi.reshape(N, N)
    for kr in range(K):
        for kc in range(K):
            win = X[np.ix_((kr * s + ar) % N, (kc * s + ar) % N)]
            out[kr * K + kc] = np.abs(M * M * np.fft.ifft2(pupil * win)) ** 2
    return PtychoData(N, M, s, chi, pupil.reshape(-1), out.reshape(-1))


def serving_requests(count: int, rate: float, seed: int = 0, n_lo: int = 100, n_hi: int = 50000,
                     deg_lo: float = 4.0, deg_hi: float = 16.0):
    """Poisson arrivals (exponential gaps at `rate` per second); sizes
    n = floor(exp(U(ln n_lo, ln n_hi))), average degree k ~ U[deg_lo, deg_hi],
    m = round(n k / 2) unit-weight edges.  Request r's graph uses seed r."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    arrivals = np.cumsum(gaps) - gaps[0]
    ns = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(np.int64)
    ks = rng.uniform(deg_lo, deg_hi, size=count)
    ms = np.minimum(np.round(ns * ks / 2).astype(np.int64), ns * (ns - 1) // 2)
    return [dict(id=r, arrival_s=float(arrivals[r]), n=int(ns[r]), m=int(ms[r]), seed=r)
            for r in range(count)]


def config_graph(name: str, seed: int = 0) -> Graph:
    """Graphs of the MaxCut workloads, by name.

    er800       : G(800, 19176), unit weights (smallest Gset shape)
    er2p20      : G(2^20, 3 * 2^20), +/-1 weights (average degree 6)
    torus2p23   : 2048 x 4096 torus + 10% long-range edges, +/-1 weights
    """
    if name == "er800":
        return er_graph(800, 19176, seed, "unit")
    if name == "er2p20":
        n = 1 << 20
        return er_graph(n, 3 * n, seed, "pm1")
    if name == "torus2p23":
        return torus_longrange_graph(2048, 4096, 0.1, seed, "pm1")
    raise KeyError(name)
