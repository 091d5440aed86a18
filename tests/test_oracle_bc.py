"""Pins of the oracle's boundary conditions (CPU only)."""
import numpy as np
import pytest

from paper_2308_06605_gb300 import inputs as I
from oracle import gas
from oracle.hexfr import HexFR

G = 1.4


def _walled_box(n, kind_lo, kind_hi, lo=(0.0, 0.0, 0.0), hi=(2.0, 1.0, 1.0), **kw):
    return I.hex_box_mesh(n, lo=lo, hi=hi, periodic=(False, True, True),
                          wall_tags={1: kind_lo, 2: kind_hi}, **kw)


@pytest.mark.parametrize("p", [3, 4])
def test_polynomial_exactness_with_dirichlet(p):
    """rho = 1, u = a + b x, p = P0: all fluxes are polynomials of degree <= 3 in x, so the
    residual equals -div(F - F_v) exactly at the solution points."""
    a, b, P0, mu = 0.3, 0.2, 2.0, 0.05
    lo, hi = (0.0, 0.0, 0.0), (1.5, 1.0, 1.0)
    state = lambda X: I.conserved(np.ones_like(X), a + b * X, 0 * X, 0 * X, P0 * np.ones_like(X), G)  # noqa: E731
    d = _walled_box((3, 2, 2), (I.BC_DIRICHLET, tuple(state(np.array(lo[0])))),
                    (I.BC_DIRICHLET, tuple(state(np.array(hi[0])))), lo=lo, hi=hi)
    phys = I.Physics(gamma=G, R=1.0, mu=mu, Pr=0.71, viscous=1)
    m = HexFR(d, phys, p)
    X = m.x[..., 0]
    Q = state(X)
    R = m.residual(Q)
    u = a + b * X
    want = np.zeros_like(Q)
    want[..., 0] = -b
    want[..., 1] = -2 * b * u
    want[..., 4] = -(G * P0 * b / (G - 1) + 1.5 * b * u * u) + 4.0 / 3.0 * mu * b * b
    np.testing.assert_allclose(R, want, rtol=0, atol=1e-11 * np.abs(want).max())   # round-off, N^2 growth


@pytest.mark.parametrize("p", [2, 3])
def test_quiescent_isothermal_walls_are_steady(p):
    Tw, rho = 1.3, 0.8
    d = _walled_box((3, 2, 2), (I.BC_WALL_ISOTHERMAL, (Tw,)), (I.BC_WALL_ISOTHERMAL, (Tw,)),
                    seed=p, rotate=True, perturb=0.1)
    phys = I.Physics(gamma=G, R=1.0, mu=0.02, Pr=0.71, viscous=1)
    m = HexFR(d, phys, p)
    one = np.ones(m.x.shape[:2])
    Q = I.conserved(rho * one, 0 * one, 0 * one, 0 * one, rho * 1.0 * Tw * one, G)
    R = m.residual(Q)
    assert np.abs(R).max() < 1e-12


@pytest.mark.parametrize("p", [2, 3])
def test_characteristic_inflow_outflow_free_stream(p):
    """A uniform subsonic stream whose total conditions and static pressure are imposed is steady."""
    rho, U, pr = 1.1, 0.35, 1.0 / G
    Rg = 1.0
    T = pr / (rho * Rg)
    cp = G * Rg / (G - 1)
    T0 = T + U * U / (2 * cp)
    p0 = pr * (T0 / T) ** (G / (G - 1))
    d = _walled_box((3, 2, 2), (I.BC_CHAR_INFLOW, (p0, T0, 1.0, 0.0, 0.0)), (I.BC_CHAR_OUTFLOW, (pr,)),
                    seed=p, rotate=True)
    phys = I.Physics(gamma=G, R=Rg, mu=0.01, Pr=0.71, viscous=1)
    m = HexFR(d, phys, p)
    one = np.ones(m.x.shape[:2])
    Q = I.conserved(rho * one, U * one, 0 * one, 0 * one, pr * one, G)
    R = m.residual(Q)
    F = np.abs(gas.inviscid_flux(Q, G)).max()
    assert np.abs(R).max() < 1e-12 * F / m.h.min()


def test_mass_conserved_in_walled_box():
    d = I.hex_box_mesh((3, 3, 3), hi=(1.0, 1.0, 1.0), periodic=(False, False, False),
                       wall_tags={t: (I.BC_WALL_ISOTHERMAL, (1.0,)) for t in range(1, 7)},
                       seed=4, perturb=0.1, rotate=True)
    phys = I.Physics(gamma=G, R=1.0, mu=0.02, Pr=0.71, viscous=1)
    m = HexFR(d, phys, 3)
    X = m.x
    rho = 1 + 0.1 * np.sin(3 * X[..., 0]) * np.cos(2 * X[..., 1])
    u = 0.1 * np.sin(np.pi * X[..., 1]) * np.sin(np.pi * X[..., 2])
    v = 0.05 * np.cos(X[..., 0] + X[..., 2])
    Q = I.conserved(rho, u, v, 0 * u, 1.0 + 0.05 * np.cos(X[..., 2]), G)
    R = m.residual(Q)
    s = abs(m.integrate(R)[0])
    a = np.einsum('m,em,em->', m.W, m.detJ, np.abs(R[..., 0]))
    assert s <= 1e-12 * a


def test_orientation_invariance_with_walls():
    phys = I.Physics(gamma=G, R=1.0, mu=0.02, Pr=0.71, viscous=1)
    kinds = ((I.BC_WALL_ISOTHERMAL, (1.1,)), (I.BC_CHAR_OUTFLOW, (0.7,)))
    ma = HexFR(_walled_box((3, 2, 2), *kinds), phys, 3)
    mb = HexFR(_walled_box((3, 2, 2), *kinds, seed=3, rotate=True, shuffle=True), phys, 3)
    def state(X):
        return I.conserved(1 + 0.1 * np.sin(X[..., 0]), 0.2 * np.cos(X[..., 1] * 2 * np.pi), 0.1 + 0 * X[..., 0],
                           0.05 * np.sin(2 * np.pi * X[..., 2]), 0.7 + 0.02 * X[..., 0], G)
    Ra, Rb = ma.residual(state(ma.x)), mb.residual(state(mb.x))
    from scipy.spatial import cKDTree
    idx = cKDTree(mb.x.reshape(-1, 3)).query(ma.x.reshape(-1, 3))[1]
    np.testing.assert_allclose(Rb.reshape(-1, 5)[idx], Ra.reshape(-1, 5), rtol=0, atol=1e-12 * np.abs(Ra).max())
