"""Pins of the oracles' energy-stable correction family (Vincent, Castonguay & Jameson 2011; the
paper's section "FR Algorithm" takes its c = 0 member), CPU only.

- Defining relation of the family, checked with numpy's Legendre class: for every phi of degree
  <= p, int phi g_R' dx + c phi^(p) g_R^(p+1) = phi(1); and g_R(1) = 1, g_R(-1) = 0.
- Named members in closed form: c_SD gives g_R = (1 + x) P_p / 2, c_HU gives Huynh's blend
  (p R_{p+1} + (p + 1) R_p) / (2p + 1) of right Radau polynomials R_k = (P_k + P_{k-1}) / 2.
- 1D linear advection, upwind flux: the FR scheme with c_SD equals an independently written
  spectral-difference scheme (flux points -1, the zeros of P_p, +1); and for any c in the
  family the energy E_c = sum_e h/2 [int u^2 + c (d^p u / dxi^p)^2] obeys the exact identity
  dE_c/dt = -|a| sum over interfaces of the squared jump.
- 3D oracles with c != 0: free stream, discrete conservation, polynomial exactness (continuous
  fluxes of degree <= p: every correction term vanishes), the hexahedral and the mixed-element
  oracles agree (BR2 and LDG, walls), and c is live.
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as L

from oracle import basis
from oracle.fr1d import residual_advection
from oracle.hexfr import HexFR
from oracle.mixedfr import MixedFR
from paper_2308_06605_gb300 import inputs as I

from helpers import vcjh_c

G = 1.4


def _apf(p):
    """a_p p! with a_p the leading coefficient of P_p."""
    return math.factorial(2 * p) / (2.0 ** p * math.factorial(p))


c_named = vcjh_c


MEMBERS = ["dg", "sd", "hu", "neg", "big"]


@pytest.mark.parametrize("which", MEMBERS)
@pytest.mark.parametrize("p", range(1, 8))
def test_defining_relation(p, which):
    c = c_named(p, which)
    N = p + 1
    xs = np.cos(np.linspace(0.0, np.pi, p + 2))
    g = L.Legendre.fit(xs, basis.correction_right(N, xs, c), p + 1, domain=[-1, 1])
    xq, wq = L.leggauss(p + 3)
    assert abs(g(1.0) - 1.0) < 1e-13 and abs(g(-1.0)) < 1e-13
    gp1 = g.deriv(p + 1)(0.0)
    for k in range(p + 1):
        phi = L.Legendre.basis(k)
        term = c * phi.deriv(p)(0.0) * gp1 if p >= 1 else 0.0
        lhs = np.sum(wq * phi(xq) * g.deriv()(xq)) + term
        assert abs(lhs - phi(1.0)) <= 1e-12 * (1.0 + abs(term)), (k, lhs, phi(1.0))
    # the derivative the schemes use is the derivative of that polynomial
    x, _ = basis.gauss_legendre(N)
    np.testing.assert_allclose(basis.correction_right_derivative(N, x, c), g.deriv()(x), rtol=0, atol=1e-11)
    b = basis.Basis1D(p, c)
    np.testing.assert_allclose(b.h_minus, b.h_plus[::-1], rtol=0, atol=1e-12)
    assert abs(np.sum(b.weights * b.h_plus) - 1.0) < 1e-12      # integral of g_R' = g_R(1) - g_R(-1)


@pytest.mark.parametrize("p", range(1, 8))
def test_named_members_closed_forms(p):
    N = p + 1
    x = np.linspace(-1.0, 1.0, 13)
    P = [L.Legendre.basis(k) for k in range(p + 2)]
    R = {k: (lambda k: (lambda t: 0.5 * (P[k](t) + P[k - 1](t))))(k) for k in range(1, p + 2)}
    np.testing.assert_allclose(basis.correction_right(N, x, 0.0), R[p + 1](x), rtol=0, atol=1e-14)
    np.testing.assert_allclose(basis.correction_right(N, x, c_named(p, "sd")), 0.5 * (1 + x) * P[p](x),
                               rtol=0, atol=1e-14)
    hu = (p * R[p + 1](x) + (p + 1) * R[p](x)) / (2 * p + 1)
    np.testing.assert_allclose(basis.correction_right(N, x, c_named(p, "hu")), hu, rtol=0, atol=1e-14)


def test_outside_the_family_raises():
    for p in (1, 3, 6):
        c_minus = -2.0 / ((2 * p + 1) * _apf(p) ** 2)
        with pytest.raises(ValueError):
            basis.Basis1D(p, c_minus * (1 + 1e-9))
        with pytest.raises(ValueError):
            basis.Basis1D(p, 1.5 * c_minus)
        basis.Basis1D(p, 0.99 * c_minus)


def _sd_residual(u, a, h, p):
    """Spectral difference for u_t + a u_x = 0, written independently of the FR oracle: the flux
    polynomial of degree p + 1 through the flux points -1, zeros of P_p, +1 takes the upwind
    common flux at the ends and a * u_h at the interior points; du/dt = -(2/h) dF/dxi."""
    K, N = u.shape
    xs, _ = L.leggauss(N)
    yi = L.leggauss(p)[0] if p >= 1 else np.zeros(0)
    y = np.concatenate([[-1.0], yi, [1.0]])
    out = np.zeros_like(u)
    polys = [L.Legendre.fit(xs, u[e], p, domain=[-1, 1]) for e in range(K)]
    left = np.array([q(-1.0) for q in polys])
    right = np.array([q(1.0) for q in polys])
    for e in range(K):
        if a >= 0:
            fl, fr = a * right[e - 1], a * right[e]
        else:
            fl, fr = a * left[e], a * left[(e + 1) % K]
        fv = np.concatenate([[fl], a * polys[e](yi), [fr]])
        F = L.Legendre.fit(y, fv, p + 1, domain=[-1, 1])
        out[e] = -(2.0 / h) * F.deriv()(xs)
    return out


@pytest.mark.parametrize("a", [0.9, -1.3])
@pytest.mark.parametrize("p", range(1, 8))
def test_sd_member_equals_spectral_difference(p, a):
    rng = np.random.default_rng(10 + p)
    K, h = 6, 0.41
    u = rng.standard_normal((K, p + 1))
    fr = residual_advection(u, a, h, p, c_named(p, "sd"))
    sd = _sd_residual(u, a, h, p)
    np.testing.assert_allclose(fr, sd, rtol=0, atol=1e-10 * np.abs(sd).max())
    # and c = 0 (DG) is a different scheme
    assert np.abs(residual_advection(u, a, h, p, 0.0) - sd).max() > 1e-3 * np.abs(sd).max()


def _energy_rate(u, r, h, p, c):
    x, w = basis.gauss_legendre(p + 1)
    rate = 0.0
    for ue, re in zip(u, r):
        du = L.Legendre.fit(x, ue, p, domain=[-1, 1]).deriv(p)(0.0)
        dr = L.Legendre.fit(x, re, p, domain=[-1, 1]).deriv(p)(0.0)
        rate += h / 2 * (2 * np.sum(w * ue * re) + 2 * c * du * dr)
    return rate


@pytest.mark.parametrize("which", MEMBERS)
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_energy_identity_1d(p, which):
    c = c_named(p, which)
    rng = np.random.default_rng(p)
    K, h = 5, 0.3
    x, _ = basis.gauss_legendre(p + 1)
    lm = basis.lagrange_values(x, [-1.0])[0]
    lp = basis.lagrange_values(x, [1.0])[0]
    for a in (1.1, -0.8):
        u = rng.standard_normal((K, p + 1))
        r = residual_advection(u, a, h, p, c)
        jumps = u @ lp - np.roll(u @ lm, -1)          # u_R of element e minus u_L of element e+1
        want = -abs(a) * np.sum(jumps ** 2)
        got = _energy_rate(u, r, h, p, c)
        scale = abs(want) + abs(_energy_rate(u, r, h, p, 0.0))
        assert abs(got - want) <= 1e-10 * scale, (got, want)
        if which != "dg":
            # the plain L2 energy is not the conserved-or-dissipated one when c != 0
            assert abs(_energy_rate(u, r, h, p, 0.0) - want) > 1e-6 * scale


def _state(X):
    return I.tgv_state(X, Ma=0.2, perturb=1e-2, seed=3)


@pytest.mark.parametrize("which", ["sd", "hu", "neg"])
@pytest.mark.parametrize("p", [2, 3])
def test_hex_oracle_free_stream_conservation(p, which):
    ph = I.tgv_physics(Ma=0.3, Re=200.0)
    ph.vcjh_c = c_named(p, which)
    m = HexFR(I.hex_box_mesh((3, 3, 2), seed=2, perturb=0.1, rotate=True, shuffle=True), ph, p)
    assert np.abs(m.residual(I.uniform_state(m.x.shape[:2]))).max() <= 1e-12
    R = m.residual(_state(m.x))
    s = np.abs(m.integrate(R))
    assert np.all(s <= 1e-12 * np.einsum('m,em,emv->v', m.W, m.detJ, np.abs(R)))
    ph.vcjh_c = 0.0
    R0 = HexFR(I.hex_box_mesh((3, 3, 2), seed=2, perturb=0.1, rotate=True, shuffle=True), ph, p).residual(_state(m.x))
    assert np.abs(R - R0).max() > 1e-6 * np.abs(R0).max()


@pytest.mark.parametrize("viscous", [1, 2])
def test_polynomial_exactness(viscous):
    a, b, P0, mu = 0.3, 0.2, 2.0, 0.05
    lo, hi = (0.0, 0.0, 0.0), (1.5, 1.0, 1.0)

    def state(X):
        return I.conserved(np.ones_like(X), a + b * X, 0 * X, 0 * X, P0 * np.ones_like(X), G)
    d = I.hex_box_mesh((3, 2, 2), lo=lo, hi=hi, periodic=(False, True, True), seed=1, rotate=True,
                       wall_tags={1: (I.BC_DIRICHLET, tuple(state(np.array(lo[0])))),
                                  2: (I.BC_DIRICHLET, tuple(state(np.array(hi[0]))))})
    p = 3
    ph = I.Physics(gamma=G, R=1.0, mu=mu, Pr=0.71, viscous=viscous, vcjh_c=c_named(p, "hu"))
    m = HexFR(d, ph, p)
    r = m.residual(state(m.x[..., 0]))
    u = a + b * m.x[..., 0]
    want = np.zeros(r.shape)
    want[..., 0] = -b
    want[..., 1] = -2 * b * u
    want[..., 4] = -(G * P0 * b / (G - 1) + 1.5 * b * u * u) + 4.0 / 3.0 * mu * b * b
    np.testing.assert_allclose(r, want, rtol=0, atol=1e-11 * 2.0)


@pytest.mark.parametrize("viscous,walls", [(1, False), (1, True), (2, True)])
def test_hex_and_mixed_oracles_agree(viscous, walls):
    p = 3
    if walls:
        d = I.hex_box_mesh((3, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, True), seed=3, rotate=True,
                           perturb=0.1, wall_tags={1: (I.BC_WALL_ISOTHERMAL, (1.1,)), 2: (I.BC_CHAR_OUTFLOW, (0.7,))})
        ph = I.Physics(gamma=G, R=1.0, mu=0.02, Pr=0.71, viscous=viscous)
    else:
        d = I.hex_box_mesh((3, 3, 2), seed=4, rotate=True, shuffle=True, perturb=0.1)
        ph = I.tgv_physics(Ma=0.2, Re=300.0)
        ph.viscous = viscous
    ph.vcjh_c = c_named(p, "sd")
    mh, mm = HexFR(d, ph, p), MixedFR(d, ph, p)
    X = mh.x
    Q = I.conserved(1 + 0.1 * np.sin(X[..., 0]), 0.2 + 0.1 * np.cos(X[..., 1]), 0.1 + 0 * X[..., 0],
                    0.05 * np.sin(2 * X[..., 2]), 0.7 + 0.02 * X[..., 0], G) if walls else _state(X)
    R1 = mh.residual(Q)
    R2 = mm.residual([Q, np.zeros((0, mm.types[1].Np, 5))])[0]
    np.testing.assert_allclose(R2, R1, rtol=0, atol=1e-13 * np.abs(R1).max())


def test_mixed_oracle_rejects_prisms_with_c():
    ph = I.tgv_physics(Ma=0.2, Re=300.0)
    ph.vcjh_c = 0.01
    with pytest.raises(ValueError):
        MixedFR(I.hex_box_mesh((2, 2, 2), prisms="checker", seed=1), ph, 2)
