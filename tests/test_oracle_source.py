"""Pins of the oracle's source term S (CPU): a sponge whose reference is the state itself adds
nothing; the body force's integral is the total momentum / work source (discrete conservation
with forcing); a constant sponge on a uniform flow gives the exact relaxation dQ/dt =
-sigma (Q - Q_ref); the parts superpose."""
import numpy as np

from oracle.mixedfr import MixedFR
from paper_2308_06605_gb300 import inputs as I


def _mesh():
    d = I.hex_box_mesh((3, 3, 2), prisms="checker", seed=2, rotate=True, perturb=0.1)
    return MixedFR(d, I.tgv_physics(Ma=0.3, Re=200.0), 3)


def test_sponge_on_own_state_is_zero_and_parts_superpose():
    m = _mesh()
    Qs = [I.tgv_state(x, Ma=0.3, perturb=1e-2, seed=1) for x in m.x]
    R0 = m.residual(Qs)
    sig = [0.5 + 0.3 * np.sin(x[..., 0]) for x in m.x]
    m.set_source(sigma=sig, Q_ref=[q.copy() for q in Qs])
    for a, b in zip(m.residual(Qs), R0):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-14 * np.abs(b).max())
    ref = [q * 1.01 for q in Qs]
    m.set_source(accel=(0.1, -0.2, 0.05), sigma=sig, Q_ref=ref)
    Rb = m.residual(Qs)
    m.set_source(accel=(0.1, -0.2, 0.05))
    Ra = m.residual(Qs)
    m.set_source(sigma=sig, Q_ref=ref)
    Rs = m.residual(Qs)
    for b, a, s, r0 in zip(Rb, Ra, Rs, R0):
        np.testing.assert_allclose(b - r0, (a - r0) + (s - r0), rtol=0, atol=1e-12 * np.abs(r0).max())


def test_body_force_integral_is_total_source():
    m = _mesh()
    g = np.array([0.3, -0.1, 0.2])
    Qs = [I.tgv_state(x, Ma=0.3, perturb=1e-2, seed=3) for x in m.x]
    m.set_source(accel=g)
    R = m.residual(Qs)
    total = m.integrate(R)
    mass = sum(np.einsum('m,em,em->', t.W, dJ, Q[..., 0]) for t, dJ, Q in zip(m.types, m.detJ, Qs))
    mom = sum(np.einsum('m,em,emj->j', t.W, dJ, Q[..., 1:4]) for t, dJ, Q in zip(m.types, m.detJ, Qs))
    scale = sum(np.einsum('m,em,emv->v', t.W, dJ, np.abs(r)) for t, dJ, r in zip(m.types, m.detJ, R))
    assert abs(total[0]) <= 1e-12 * scale[0]
    np.testing.assert_allclose(total[1:4], mass * g, rtol=0, atol=1e-12 * scale[1:4].max())
    assert abs(total[4] - mom @ g) <= 1e-12 * scale[4]


def test_uniform_flow_relaxes_exactly():
    m = _mesh()
    U = [I.uniform_state(x.shape[:2]) for x in m.x]
    ref = [I.uniform_state(x.shape[:2], rho=1.2, vel=(0.1, 0.0, 0.0)) for x in m.x]
    m.set_source(sigma=[2.0 * np.ones(x.shape[:2]) for x in m.x], Q_ref=ref)
    for R, q, r in zip(m.residual(U), U, ref):
        np.testing.assert_allclose(R, -2.0 * (q - r), rtol=0, atol=1e-12)
