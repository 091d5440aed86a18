"""Pins of the oracle's Roe flux (CPU): what Roe's construction fixes independently of its code.

- Property U: with the signed eigenvalues, sum_k lambda_k alpha_k r_k |n| = (F(QR) - F(QL)) . n
  exactly for any two states (the Roe-averaged Jacobian linearises the flux jump).
- Consistency F(Q, Q) = F(Q) . n; conservation F(QL, QR, n) = -F(QR, QL, -n).
- Supersonic upwinding: all waves to the right (u.n^ > 1.2 c) gives F(QL) . n.
- A stationary contact (density jump, equal velocity zero and pressure) passes without dissipation.
- Rotational invariance of the momentum components.
And of the FR residual with the Roe flux: free-stream preservation and discrete conservation.
"""
import numpy as np
import pytest

from oracle import gas
from oracle.hexfr import HexFR
from paper_2308_06605_gb300 import inputs as I

G = 1.4


def _states(rng, n, mach=0.8):
    rho = rng.uniform(0.5, 2.0, n)
    u = rng.normal(0, mach, (n, 3))
    p = rng.uniform(0.5, 2.0, n)
    return I.conserved(rho, u[:, 0], u[:, 1], u[:, 2], p, G)


def _fdot(Q, n):
    return np.einsum('...jv,...j->...v', gas.inviscid_flux(Q, G), n)


def test_property_u():
    rng = np.random.default_rng(0)
    QL, QR = _states(rng, 200), _states(rng, 200)
    n = rng.normal(size=(200, 3)) * rng.uniform(0.3, 3.0, (200, 1))
    lhs = gas.roe_dissipation(QL, QR, n, G, absolute=False)
    rhs = _fdot(QR, n) - _fdot(QL, n)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12 * np.abs(rhs).max())


def test_consistency_and_conservation():
    rng = np.random.default_rng(1)
    QL, QR = _states(rng, 100), _states(rng, 100)
    n = rng.normal(size=(100, 3))
    np.testing.assert_allclose(gas.roe(QL, QL, n, G), _fdot(QL, n), rtol=0, atol=1e-13 * 10)
    np.testing.assert_allclose(gas.roe(QL, QR, n, G), -gas.roe(QR, QL, -n, G), rtol=0, atol=1e-12)


def test_supersonic_upwinding():
    rng = np.random.default_rng(2)
    k = 100
    n = rng.normal(size=(k, 3))
    nh = n / np.linalg.norm(n, axis=1)[:, None]
    rho = rng.uniform(0.8, 1.2, (2, k))
    p = rng.uniform(0.8, 1.2, (2, k))
    c = np.sqrt(G * p / rho)
    u = (2.0 * c.max(axis=0))[None, :, None] * nh[None] + rng.normal(0, 0.05, (2, k, 3))
    QL = I.conserved(rho[0], u[0, :, 0], u[0, :, 1], u[0, :, 2], p[0], G)
    QR = I.conserved(rho[1], u[1, :, 0], u[1, :, 1], u[1, :, 2], p[1], G)
    np.testing.assert_allclose(gas.roe(QL, QR, n, G), _fdot(QL, n), rtol=0, atol=1e-12 * 50)


def test_stationary_contact():
    n = np.array([[0.3, -1.2, 0.5]])
    QL = I.conserved(np.array([1.0]), 0 * n[:, 0], 0 * n[:, 0], 0 * n[:, 0], np.array([1.3]), G)
    QR = I.conserved(np.array([0.4]), 0 * n[:, 0], 0 * n[:, 0], 0 * n[:, 0], np.array([1.3]), G)
    want = np.zeros((1, 5))
    want[0, 1:4] = 1.3 * n[0]
    np.testing.assert_allclose(gas.roe(QL, QR, n, G), want, rtol=0, atol=1e-14)
    # Rusanov, by contrast, smears it.
    assert np.abs(gas.rusanov(QL, QR, n, G) - want).max() > 1e-2


def test_rotational_invariance():
    rng = np.random.default_rng(3)
    QL, QR = _states(rng, 50), _states(rng, 50)
    n = rng.normal(size=(50, 3))
    A, _ = np.linalg.qr(rng.normal(size=(3, 3)))

    def rot(Q):
        out = Q.copy()
        out[:, 1:4] = Q[:, 1:4] @ A.T
        return out
    F = gas.roe(QL, QR, n, G)
    Fr = gas.roe(rot(QL), rot(QR), n @ A.T, G)
    np.testing.assert_allclose(Fr, rot(F), rtol=0, atol=1e-12)


@pytest.mark.parametrize("p", [2, 3])
def test_residual_with_roe_free_stream_and_conservation(p):
    d = I.hex_box_mesh((3, 3, 2), seed=p, perturb=0.15, rotate=True, shuffle=True)
    ph = I.tgv_physics(Ma=0.3, Re=200.0)
    ph.inviscid_flux = 1
    m = HexFR(d, ph, p)
    U = I.uniform_state(m.x.shape[:2])
    assert np.abs(m.residual(U)).max() <= 1e-12
    Q = I.tgv_state(m.x, Ma=0.3, perturb=1e-2, seed=p)
    R = m.residual(Q)
    s = np.abs(m.integrate(R))
    a = np.einsum('m,em,emv->v', m.W, m.detJ, np.abs(R))
    assert np.all(s <= 1e-12 * a), s / a
    # Roe and Rusanov residuals differ (the switch is live) but agree to the dissipation's size.
    ph.inviscid_flux = 0
    R0 = HexFR(d, ph, p).residual(Q)
    assert 0 < np.abs(R - R0).max() < 0.2 * np.abs(R0).max()
