"""Pins for the oracle's random streams (Philox4x32-10 + Box-Muller)."""
import os

import numpy as np
import pytest
from scipy import stats

from oracle.philox import (PURPOSE_LANCZOS, PURPOSE_OMEGA, gaussian_matrix, gaussian_vector,
                           normals, philox4x32_10)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([int(x, 16) for x in line.split()])
    return rows


@pytest.mark.parametrize("row", _kat())
def test_philox_known_answers(row):
    out = philox4x32_10(*row[:6])
    assert [int(x) for x in out] == row[6:]


def test_normals_are_standard_normal():
    x = normals(7, PURPOSE_LANCZOS, 3, 0, 200_000)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01
    assert stats.kstest(x, "norm").pvalue > 1e-3
    # the two Box-Muller outputs of one pair are uncorrelated
    assert abs(np.corrcoef(x[0::2], x[1::2])[0, 1]) < 0.01


def test_streams_independent_and_addressable():
    a = normals(0, PURPOSE_LANCZOS, 1, 0, 1000)
    b = normals(0, PURPOSE_LANCZOS, 2, 0, 1000)
    c = normals(0, PURPOSE_OMEGA, 1, 0, 1000)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.15 and abs(np.corrcoef(a, c)[0, 1]) < 0.15
    # random access: a sub-range equals the slice of the full stream
    np.testing.assert_array_equal(normals(0, PURPOSE_LANCZOS, 1, 0, 10, start=501), a[501:511])


def test_complex_and_matrix_layout():
    g = normals(5, PURPOSE_OMEGA, 0, 2, 24)
    Z = gaussian_matrix(5, PURPOSE_OMEGA, 2, 4, 3, True)
    np.testing.assert_array_equal(Z.reshape(-1), g[0::2] + 1j * g[1::2])
    R = gaussian_matrix(5, PURPOSE_OMEGA, 2, 4, 3, False)
    np.testing.assert_array_equal(R.reshape(-1), g[:12])
    v = gaussian_vector(5, PURPOSE_OMEGA, 0, 2, 12, False)
    np.testing.assert_array_equal(v, g[:12])
