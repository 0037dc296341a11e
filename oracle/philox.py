"""Philox4x32-10 and Box-Muller Gaussian streams (oracle side).

The paper draws its random quantities with MATLAB ``randn`` (Alg. 4.1, first
line; Alg. 5.1 ``NystromSketch.Init``) and does not fix a generator.  Both this
oracle and the CUDA library implement the counter-based generator Philox4x32
with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
as 1, 2, 3", SC'11), each from that published definition, so that they draw
identical numbers without sharing code.

Stream layout (shared convention, stated here and in the C header):
  normal number m of stream (seed, purpose, t, instance) is output (m & 1) of
  Box-Muller applied to Philox4x32-10 with
      counter = (m >> 1, t, purpose, instance)   key = (seed & 0xffffffff, seed >> 32)
  The four 32-bit outputs x0..x3 give two 53-bit uniforms on (0, 1):
      u = ((x_a >> 5) * 2^26 + (x_b >> 6) + 0.5) / 2^53   for (a, b) = (0, 1), (2, 3)
  and Box-Muller gives  r = sqrt(-2 ln u1),  normal0 = r cos(2 pi u2),
  normal1 = r sin(2 pi u2).
Complex standard normals (footnote to Section 5.1: real and imaginary parts
independent N(0,1)) take normal 2k as the real part of entry k and 2k+1 as its
imaginary part.
"""
from __future__ import annotations

import numpy as np

PURPOSE_OMEGA = 1    # Nystrom test matrix Omega (Alg. 5.1 Init)
PURPOSE_LANCZOS = 2  # random start vector of ApproxMinEvec (Alg. 4.1)

_M32 = np.uint64(0xFFFFFFFF)
_MUL0 = np.uint64(0xD2511F53)
_MUL1 = np.uint64(0xCD9E8D57)
_WEYL0 = np.uint64(0x9E3779B9)
_WEYL1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit values (held in uint64).

    One round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (64-bit products),
    new counter = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by
    the Weyl constants between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _M32 for x in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for r in range(10):
        if r:
            k0 = (k0 + _WEYL0) & _M32
            k1 = (k1 + _WEYL1) & _M32
        p0 = _MUL0 * c0
        p1 = _MUL1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _M32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _M32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def _uniform53(a, b):
    a = (a >> np.uint64(5)).astype(np.float64)
    b = (b >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b + 0.5) / 9007199254740992.0


def normals(seed: int, purpose: int, t: int, instance: int, count: int, start: int = 0) -> np.ndarray:
    """Normals start .. start+count-1 of stream (seed, purpose, t, instance)."""
    if count == 0:
        return np.zeros(0)
    m = np.arange(start, start + count, dtype=np.uint64)
    pair = m >> np.uint64(1)
    if int(pair[-1]) >= 2**32:
        raise ValueError("stream index exceeds 2^33")
    x0, x1, x2, x3 = philox4x32_10(pair, np.uint64(t), np.uint64(purpose), np.uint64(instance),
                                   seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u1 = _uniform53(x0, x1)
    u2 = _uniform53(x2, x3)
    r = np.sqrt(-2.0 * np.log(u1))
    theta = 2.0 * np.pi * u2
    odd = (m & np.uint64(1)).astype(bool)
    return np.where(odd, r * np.sin(theta), r * np.cos(theta))


def gaussian_vector(seed: int, purpose: int, t: int, instance: int, n: int, complex_: bool) -> np.ndarray:
    """randn(n, 1) of the given stream; complex entries use normals (2k, 2k+1)."""
    if complex_:
        g = normals(seed, purpose, t, instance, 2 * n)
        return g[0::2] + 1j * g[1::2]
    return normals(seed, purpose, t, instance, n)


def gaussian_matrix(seed: int, purpose: int, instance: int, n: int, R: int, complex_: bool) -> np.ndarray:
    """randn(n, R): entry (i, c) is stream entry i*R + c (row-major), t = 0."""
    return gaussian_vector(seed, purpose, 0, instance, n * R, complex_).reshape(n, R)
