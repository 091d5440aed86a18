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


def _prim(Q, g):
    rho = Q[..., 0]
    u = Q[..., 1:4] / rho[..., None]
    p = (g - 1.0) * (Q[..., 4] - 0.5 * rho * np.sum(u * u, axis=-1))
    return rho, u, p


def _random_subsonic(rng, n, g, Rg):
    rho = rng.uniform(0.8, 1.2, n)
    p = rng.uniform(0.7, 1.3, n)
    c = np.sqrt(g * p / rho)
    u = rng.normal(size=(n, 3)) * 0.15 * c[:, None]
    Q = np.concatenate([rho[:, None], rho[:, None] * u, (p / (g - 1.0) + 0.5 * rho * np.sum(u * u, -1))[:, None]], 1)
    nrm = rng.normal(size=(n, 3)) * rng.uniform(0.5, 2.0, (n, 1))
    return Q, nrm


def test_characteristic_outflow_state_obeys_its_defining_relations():
    """Static pressure imposed; entropy p / rho^gamma, tangential velocity and the outgoing
    Riemann invariant u.n + 2c/(gamma-1) carried from the interior (checked with formulas
    written here); imposing the interior's own pressure returns the interior state."""
    from oracle.hexfr import boundary_states
    g, Rg = 1.4, 287.0 / 1000.0
    rng = np.random.default_rng(3)
    Qm, n = _random_subsonic(rng, 64, g, Rg)
    nh = n / np.linalg.norm(n, axis=-1, keepdims=True)
    pb = 0.93
    Qg, Qi = boundary_states(I.BC_CHAR_OUTFLOW, np.array([pb, 0, 0, 0, 0, 0, 0, 0.0]), Qm, n, g, Rg)
    assert np.array_equal(Qg, Qi)
    r0, u0, p0 = _prim(Qm, g)
    rb, ub, pbb = _prim(Qg, g)
    np.testing.assert_allclose(pbb, pb, rtol=1e-13)
    np.testing.assert_allclose(pbb / rb ** g, p0 / r0 ** g, rtol=1e-12)
    tang = lambda u: u - np.sum(u * nh, -1)[:, None] * nh  # noqa: E731
    np.testing.assert_allclose(tang(ub), tang(u0), atol=1e-13)
    inv = lambda r, u, p: np.sum(u * nh, -1) + 2.0 * np.sqrt(g * p / r) / (g - 1.0)  # noqa: E731
    np.testing.assert_allclose(inv(rb, ub, pbb), inv(r0, u0, p0), rtol=1e-13)
    for k in range(4):
        Qs, _ = boundary_states(I.BC_CHAR_OUTFLOW, np.array([p0[k], 0, 0, 0, 0, 0, 0, 0.0]), Qm[k:k + 1], n[k:k + 1], g, Rg)
        np.testing.assert_allclose(Qs[0], Qm[k], rtol=1e-13, atol=1e-14)


def test_characteristic_inflow_state_obeys_isentropic_total_conditions():
    """Total temperature T0 = T + |u|^2 / (2 cp), total pressure p0 = p (T0 / T)^(gamma/(gamma-1)),
    velocity along the prescribed direction, and the outgoing invariant carried from the
    interior (formulas written here)."""
    from oracle.hexfr import boundary_states
    g, Rg = 1.4, 0.287
    cp = g * Rg / (g - 1.0)
    rng = np.random.default_rng(4)
    p0, T0, M = 1.2, 3.9, 0.3
    d = np.array([1.0, 0.3, -0.2])
    dh = d / np.linalg.norm(d)
    # Interior states: the isentropic state of (p0, T0) at Mach 0.3 along d, perturbed by ~2 %.
    nq = 64
    T = T0 / (1.0 + 0.5 * (g - 1.0) * M * M) * rng.uniform(0.98, 1.02, nq)
    pr = p0 * (T / T0) ** (g / (g - 1.0)) * rng.uniform(0.98, 1.02, nq)
    rho = pr / (Rg * T)
    u = (M * np.sqrt(g * Rg * T))[:, None] * dh[None, :] * rng.uniform(0.9, 1.1, (nq, 1)) + \
        0.02 * rng.normal(size=(nq, 3))
    Qm = np.concatenate([rho[:, None], rho[:, None] * u, (pr / (g - 1.0) + 0.5 * rho * np.sum(u * u, -1))[:, None]], 1)
    # Inflow faces: the outward normal points against the flow direction, tilted.
    n = rng.uniform(0.5, 2.0, (nq, 1)) * (-dh[None, :] + 0.3 * rng.normal(size=(nq, 3)))
    nh = n / np.linalg.norm(n, axis=-1, keepdims=True)
    Qg, Qi = boundary_states(I.BC_CHAR_INFLOW, np.array([p0, T0, *d, 0, 0, 0.0]), Qm, n, g, Rg)
    assert np.array_equal(Qg, Qi)
    rb, ub, pb = _prim(Qg, g)
    Tb = pb / (rb * Rg)
    V = np.linalg.norm(ub, axis=-1)
    np.testing.assert_allclose(Tb + V * V / (2.0 * cp), T0, rtol=1e-13)
    np.testing.assert_allclose(pb * (T0 / Tb) ** (g / (g - 1.0)), p0, rtol=1e-12)
    np.testing.assert_allclose(np.cross(ub, dh), 0.0, atol=1e-13)
    assert np.all(ub @ dh > 0)
    r0, u0, pm = _prim(Qm, g)
    inv = lambda r, u, p: np.sum(u * nh, -1) + 2.0 * np.sqrt(g * p / r) / (g - 1.0)  # noqa: E731
    np.testing.assert_allclose(inv(rb, ub, pb), inv(r0, u0, pm), rtol=1e-12)
