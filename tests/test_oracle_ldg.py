"""Pins of the oracles' LDG viscous discretisation (CPU), and of both viscous schemes against a
closed-form viscous residual.

- The hexahedral and the mixed-element oracles (independent interface code) agree with LDG,
  also with walls and characteristic boundaries.
- A polynomial state whose fluxes have degree <= p, continuous across elements: all jumps vanish
  and the residual equals the exact divergence.
- Free stream, discrete conservation (periodic) and orientation / shuffle invariance (the LDG
  switch is geometric, not tied to the element order).
- Shear wave rho = 1, p = P0, v = A sin(x): the exact residual is R_rhov = -mu A sin(x),
  R_E = mu A^2 cos(2x); both BR2 and LDG converge to it pointwise (order about p - 1).
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import gas
from oracle.hexfr import HexFR
from oracle.mixedfr import MixedFR
from paper_2308_06605_gb300 import inputs as I

G = 1.4


def _ldg(ph, tau=0.1):
    ph.viscous, ph.ldg_tau = 2, tau
    return ph


@pytest.mark.parametrize("walls", [False, True])
def test_hex_and_mixed_oracles_agree(walls):
    if walls:
        d = I.hex_box_mesh((3, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, True), seed=3, rotate=True,
                           perturb=0.1, wall_tags={1: (I.BC_WALL_ISOTHERMAL, (1.1,)), 2: (I.BC_CHAR_OUTFLOW, (0.7,))})
        ph = _ldg(I.Physics(gamma=G, R=1.0, mu=0.02, Pr=0.71, viscous=1))
    else:
        d = I.hex_box_mesh((3, 3, 2), seed=4, rotate=True, shuffle=True, perturb=0.1)
        ph = _ldg(I.tgv_physics(Ma=0.2, Re=300.0))
    mh, mm = HexFR(d, ph, 3), MixedFR(d, ph, 3)
    X = mh.x
    Q = I.conserved(1 + 0.1 * np.sin(X[..., 0]), 0.2 + 0.1 * np.cos(X[..., 1]), 0.1 + 0 * X[..., 0],
                    0.05 * np.sin(2 * X[..., 2]), 0.7 + 0.02 * X[..., 0], G) if walls else \
        I.tgv_state(X, Ma=0.2, perturb=1e-2, seed=2)
    R1 = mh.residual(Q)
    R2 = mm.residual([Q, np.zeros((0, mm.types[1].Np, 5))])[0]
    np.testing.assert_allclose(R2, R1, rtol=0, atol=1e-13 * np.abs(R1).max())
    # and LDG differs from BR2 (the scheme switch is live)
    ph.viscous = 1
    assert np.abs(HexFR(d, ph, 3).residual(Q) - R1).max() > 1e-6 * np.abs(R1).max()


@pytest.mark.parametrize("prisms", [None, "checker"])
def test_polynomial_exactness(prisms):
    a, b, P0, mu = 0.3, 0.2, 2.0, 0.05
    lo, hi = (0.0, 0.0, 0.0), (1.5, 1.0, 1.0)
    state = lambda X: I.conserved(np.ones_like(X), a + b * X, 0 * X, 0 * X, P0 * np.ones_like(X), G)  # noqa: E731
    d = I.hex_box_mesh((3, 2, 2), lo=lo, hi=hi, periodic=(False, True, True), prisms=prisms, seed=1, rotate=True,
                       wall_tags={1: (I.BC_DIRICHLET, tuple(state(np.array(lo[0])))),
                                  2: (I.BC_DIRICHLET, tuple(state(np.array(hi[0]))))})
    m = MixedFR(d, _ldg(I.Physics(gamma=G, R=1.0, mu=mu, Pr=0.71, viscous=1)), 3)
    for x, r in zip(m.x, m.residual([state(x[..., 0]) for x in m.x])):
        u = a + b * x[..., 0]
        want = np.zeros(r.shape)
        want[..., 0] = -b
        want[..., 1] = -2 * b * u
        want[..., 4] = -(G * P0 * b / (G - 1) + 1.5 * b * u * u) + 4.0 / 3.0 * mu * b * b
        np.testing.assert_allclose(r, want, rtol=0, atol=1e-11 * 2.0)


@pytest.mark.parametrize("p", [2, 3])
def test_free_stream_conservation_and_orientation_invariance(p):
    ph = _ldg(I.tgv_physics(Ma=0.3, Re=200.0))
    ma = HexFR(I.hex_box_mesh((3, 3, 2), seed=2, perturb=0.1), ph, p)
    mb = HexFR(I.hex_box_mesh((3, 3, 2), seed=2, perturb=0.1, rotate=True, shuffle=True), ph, p)
    assert np.abs(ma.residual(I.uniform_state(ma.x.shape[:2]))).max() <= 1e-12
    Qa = I.tgv_state(ma.x, Ma=0.3, perturb=1e-2, seed=p)
    Ra = ma.residual(Qa)
    s = np.abs(ma.integrate(Ra))
    assert np.all(s <= 1e-12 * np.einsum('m,em,emv->v', ma.W, ma.detJ, np.abs(Ra)))
    Rb = mb.residual(I.tgv_state(mb.x, Ma=0.3, perturb=1e-2, seed=p))
    ei = cKDTree(mb.x.mean(axis=1)).query(ma.x.mean(axis=1))[1]
    for e in range(ma.E):
        dd, i = cKDTree(mb.x[ei[e]]).query(ma.x[e])
        assert dd.max() < 1e-9
        np.testing.assert_allclose(Rb[ei[e]][i], Ra[e], rtol=0, atol=1e-11 * np.abs(Ra).max())


def test_switch_direction_is_live():
    d = I.hex_box_mesh((3, 3, 2), seed=6, perturb=0.1)
    ph = _ldg(I.tgv_physics(Ma=0.3, Re=200.0))
    m = HexFR(d, ph, 2)
    Q = I.tgv_state(m.x, Ma=0.3, perturb=1e-2, seed=1)
    R1 = m.residual(Q)
    saved = gas.LDG_SWITCH.copy()
    try:
        gas.LDG_SWITCH[:] = -saved
        R2 = m.residual(Q)
    finally:
        gas.LDG_SWITCH[:] = saved
    assert np.abs(R2 - R1).max() > 1e-8 * np.abs(R1).max()


@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("p", [2, 3, 4])
def test_shear_wave_residual_converges(scheme, p):
    """Pointwise residual error of the viscous operator converges like h^(p-1) (a second
    derivative of an order-(p+1) approximation); the bar is p - 1.5 on two levels."""
    A, P0, mu = 0.1, 1.0, 0.05
    errs = []
    for n in (8, 16):
        d = I.hex_box_mesh((n, 1, 1), hi=(2 * np.pi, 1.0, 1.0))
        ph = I.Physics(gamma=G, R=1.0, mu=mu, Pr=0.71, viscous=scheme, ldg_tau=0.1)
        m = HexFR(d, ph, p)
        X = m.x[..., 0]
        R = m.residual(I.conserved(np.ones_like(X), 0 * X, A * np.sin(X), 0 * X, P0 * np.ones_like(X), G))
        want = np.zeros(R.shape)
        want[..., 2] = -mu * A * np.sin(X)
        want[..., 4] = mu * A * A * np.cos(2 * X)
        errs.append(np.abs(R - want).max() / (mu * A))
    assert errs[1] < 0.8 and np.log2(errs[0] / errs[1]) > p - 1.5, errs


@pytest.mark.parametrize("p", [2, 3])
def test_penalty_dissipates_the_squared_jumps_exactly(p):
    """Changing tau only changes the penalty tau |n| (Q_0 - Q_1) of the common normal flux; with
    the DG-equivalent lifting its contribution to sum_e sum_m W |J| Q . R is exactly
    -dtau sum_faces sum_fp w_fp |n| |Q_0 - Q_1|^2 (computed here from the basis values on an
    axis-aligned periodic 4x1x1 box, where every jump is known by construction)."""
    from oracle.basis import Basis1D
    hx, hy, hz = 0.7, 1.3, 0.9
    d = I.hex_box_mesh((4, 1, 1), hi=(4 * hx, hy, hz))
    rng = np.random.default_rng(p)
    N = p + 1
    R = []
    for tau in (0.1, 0.35):
        ph = I.Physics(gamma=G, R=1.0, mu=0.03, Pr=0.71, viscous=2, ldg_tau=tau)
        m = HexFR(d, ph, p)
        if not R:
            # element e spans [e hx, (e+1) hx] with xi along +x (unrotated, unshuffled box)
            assert np.allclose(m.x[:, 0, 0], np.arange(4) * hx + hx / 2 * (1 + Basis1D(p).nodes[0]))
            Q = I.uniform_state(m.x.shape[:2]) * (1 + 0.05 * rng.standard_normal(m.x.shape[:2] + (5,)))
        R.append(m.residual(Q))
    dE = np.einsum('m,em,emv,emv->', m.W, m.detJ, Q, R[1] - R[0])
    b = Basis1D(p)
    q = Q.reshape(4, N, N, N, 5)            # [e][k][j][i][v]
    wf = np.outer(b.weights, b.weights)     # face quadrature weights over the two tangential axes
    jump2 = 0.0
    for e in range(4):                      # x faces: element e's +x trace against e+1's -x trace
        right = np.einsum('i,kjiv->kjv', b.l_plus, q[e])
        left = np.einsum('i,kjiv->kjv', b.l_minus, q[(e + 1) % 4])
        jump2 += hy * hz / 4 * np.sum(wf[:, :, None] * (right - left) ** 2)
        # y and z faces: the element meets itself through the periodic pairs
        yj = np.einsum('j,kjiv->kiv', b.l_plus, q[e]) - np.einsum('j,kjiv->kiv', b.l_minus, q[e])
        zj = np.einsum('k,kjiv->jiv', b.l_plus, q[e]) - np.einsum('k,kjiv->jiv', b.l_minus, q[e])
        jump2 += hx * hz / 4 * np.sum(wf[:, :, None] * yj ** 2) + hx * hy / 4 * np.sum(wf[:, :, None] * zj ** 2)
    want = -(0.35 - 0.1) * jump2
    assert want < 0 and abs(dE - want) <= 1e-10 * abs(want), (dE, want)
