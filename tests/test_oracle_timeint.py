"""Pins of the oracle's RK integrators (CPU): stability polynomials, orders, SSP coefficients."""
import math

import numpy as np
import pytest

from oracle import timeint as TI


def _amp(scheme, z):
    """Amplification factor on y' = lambda y at z = lambda dt (dt = 1)."""
    return TI.SCHEMES[scheme](lambda Q: [z * Q[0]], [np.array(1.0 + 0j)], 1.0)[0]


def test_rk44_and_ssprk33_stability_polynomials():
    for z in (0.3, -1.7, 0.5 + 1.2j, -2.0 - 0.4j):
        assert abs(_amp("rk44", z) - sum(z ** k / math.factorial(k) for k in range(5))) < 1e-13
        assert abs(_amp("ssprk33", z) - sum(z ** k / math.factorial(k) for k in range(4))) < 1e-13


def test_ssprk104_is_fourth_order_and_has_ssp_coefficient_six():
    # Taylor agreement to z^4: the error of the stability polynomial is O(z^5).
    errs = []
    for z in (0.2, 0.1, 0.05):
        errs.append(abs(_amp("ssprk104", z) - sum(z ** k / math.factorial(k) for k in range(5))))
    assert errs[0] / errs[1] > 25 and errs[1] / errs[2] > 25          # ~ 2^5
    # SSP coefficient 6: forward Euler keeps y' = -y positive and non-increasing for dt <= 1, the
    # scheme (a convex combination of Euler substeps of dt/6) for dt <= 6; SSPRK33 (coefficient 1)
    # for dt <= 1.
    for dt in np.linspace(0.0, 6.0, 61):
        assert -1e-12 <= _amp("ssprk104", -dt).real <= 1.0 + 1e-12
    for dt in np.linspace(0.0, 1.0, 11):
        assert -1e-12 <= _amp("ssprk33", -dt).real <= 1.0 + 1e-12


@pytest.mark.parametrize("scheme,order", [("rk44", 4), ("ssprk33", 3), ("ssprk104", 4)])
def test_convergence_order_on_a_nonlinear_system(scheme, order):
    """u' = -v + u v, v' = u - v^2 / 2: observed order against a fine reference."""
    def f(Q):
        u, v = Q
        return [-v + u * v, u - 0.5 * v * v]

    def run(n):
        Q = [np.array(0.3), np.array(-0.2)]
        for _ in range(n):
            Q = TI.SCHEMES[scheme](f, Q, 1.0 / n)
        return np.array([float(Q[0]), float(Q[1])])
    ref = run(4096)
    e1, e2 = np.abs(run(16) - ref).max(), np.abs(run(32) - ref).max()
    assert np.log2(e1 / e2) > order - 0.3
