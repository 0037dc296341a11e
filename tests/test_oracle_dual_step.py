"""Pin of the oracle's dual step size (Eq. 6.4) against the paper's other
statement of the same condition.

Eq. 6.4 bounds gamma_t ||z - b||^2 by 4 alpha^2 beta0 ||A||^2 / (t+1)^{3/2};
the CGAL iteration of App. A.3 states the bound as beta_t eta_t^2 alpha^2
||A||^2 in terms of the iteration's own schedules, beta_t = beta0 sqrt(t+1)
and eta_t = 2 / (t+1) (Alg. 6.1).  Evaluating the appendix form from those
schedules is an independent route to the number: a dropped factor 4, a wrong
exponent on t + 1 or a missing alpha^2 in the oracle fails here.  In both,
gamma_t is the largest value that also satisfies 0 <= gamma_t <= beta0.
"""
import math

import numpy as np
import pytest

from oracle.sketchycgal import dual_step


def _appendix_gamma(normsq_zb, t, alpha, beta0, normA):
    beta_t = beta0 * math.sqrt(t + 1)
    eta_t = 2.0 / (t + 1)
    bound = beta_t * eta_t ** 2 * alpha ** 2 * normA ** 2
    return beta0 if normsq_zb == 0.0 else min(beta0, bound / normsq_zb)


@pytest.mark.parametrize("seed", range(5))
def test_dual_step_matches_the_appendix_form(seed):
    rng = np.random.default_rng(seed)
    for _ in range(200):
        t = int(rng.integers(1, 100000))
        alpha = float(10 ** rng.uniform(-2, 6))
        beta0 = float(10 ** rng.uniform(-2, 2))
        normA = float(10 ** rng.uniform(-1, 3))
        normsq = float(10 ** rng.uniform(-12, 12))
        g = dual_step(normsq, t, alpha, beta0, normA)
        assert g == pytest.approx(_appendix_gamma(normsq, t, alpha, beta0, normA), rel=1e-13)


def test_dual_step_is_the_largest_admissible_value():
    t, alpha, beta0, normA = 40, 3.0, 1.0, 2.0
    bound = 4 * alpha ** 2 * beta0 * normA ** 2 / (t + 1) ** 1.5
    # a large residual: the bound binds, with equality
    g = dual_step(10.0, t, alpha, beta0, normA)
    assert g < beta0 and g * 10.0 == pytest.approx(bound, rel=1e-15)
    # a small residual: the cap beta0 binds
    assert dual_step(1e-9, t, alpha, beta0, normA) == beta0
    # z = b exactly: any gamma satisfies the bound, so the cap
    assert dual_step(0.0, t, alpha, beta0, normA) == beta0
    # the bound shrinks like (t + 1)^(-3/2)
    g1, g2 = dual_step(1e6, 99, alpha, beta0, normA), dual_step(1e6, 399, alpha, beta0, normA)
    assert g1 / g2 == pytest.approx(8.0, rel=1e-12)
