"""Pins of the oracle's triangle basis (prism layers), CPU only."""
import math

import numpy as np
import pytest

from oracle import tri


def _monomial_integral(a, b):
    """int_T r^a s^b over the reference triangle, brute force with a tensor Gauss rule on the
    collapsed square (exact for polynomials): r = (1+u)(1-s)/2 - 1."""
    x, w = np.polynomial.legendre.leggauss(12)
    U, S = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w)
    R = (1 + U) * (1 - S) / 2 - 1
    jac = (1 - S) / 2
    return float(np.sum(W * jac * R ** a * S ** b))


@pytest.mark.parametrize("p", range(1, 8))
def test_nodes_symmetric_inside_unisolvent(p):
    rs = tri.nodes(p)
    assert rs.shape[0] == (p + 1) * (p + 2) // 2
    r, s = rs[:, 0], rs[:, 1]
    assert np.all(r >= -1 - 1e-12) and np.all(s >= -1 - 1e-12) and np.all(r + s <= 1e-12)
    # symmetric under the reflection r <-> s and the rotation (r, s) -> (s, -1 - r - s)
    for img in (np.stack([s, r], 1), np.stack([-r - s - 1, r], 1)):
        d = np.linalg.norm(img[:, None, :] - rs[None, :, :], axis=-1).min(axis=1)
        assert d.max() < 1e-10
    T = tri.Tri(p)
    assert np.linalg.cond(T.V) < 1e3


@pytest.mark.parametrize("p", range(1, 8))
def test_derivatives_and_mass_exact(p):
    T = tri.Tri(p)
    r, s = T.rs[:, 0], T.rs[:, 1]
    for a in range(p + 1):
        for b in range(p + 1 - a):
            f = r ** a * s ** b
            dr = a * r ** max(a - 1, 0) * s ** b if a else 0 * r
            ds = b * r ** a * s ** max(b - 1, 0) if b else 0 * r
            np.testing.assert_allclose(T.Dr @ f, dr, atol=1e-10)
            np.testing.assert_allclose(T.Ds @ f, ds, atol=1e-10)
            # mass matrix integrates products exactly: 1^T M f = int f
            assert abs(np.ones(T.Nt) @ T.M @ f - _monomial_integral(a, b)) < 1e-12
    assert abs(np.ones(T.Nt) @ T.M @ np.ones(T.Nt) - 2.0) < 1e-13


def test_interpolation_at_edges():
    T = tri.Tri(4)
    x = np.linspace(-1, 1, 9)
    pts = np.stack([x, -np.ones_like(x)], 1)
    L = T.interp(pts)
    f = T.rs[:, 0] ** 3 - 2 * T.rs[:, 1] * T.rs[:, 0]
    np.testing.assert_allclose(L @ f, x ** 3 + 2 * x, atol=1e-12)
