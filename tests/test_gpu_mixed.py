"""Mixed-precision path (FR_PREC_MIXED) vs the FP64 oracle, through the C ABI (marked gpu).

The element operators run in double-float (FP32 hi + lo pairs, ~44-bit); the Riemann flux,
boundary states and the RK update stay FP64.  Stated error bars:
  per entry   |R_mixed - R_oracle| <= 1e-9 * S   (S: the oracle's magnitude scale of the entry)
  normwise    max|R_mixed - R_oracle| / max|R_oracle| <= 1e-6 per variable (the target)
"""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle.hexfr import HexFR

from helpers import assert_residual_parity, assert_state_parity, ensure_lib

pytestmark = pytest.mark.gpu

MIXED_ENTRY = 1e-9
MIXED_NORM = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _mixed(phys):
    ph = I.Physics(**{k: getattr(phys, k) for k in phys.__dataclass_fields__})
    ph.precision = 1
    return ph


def _check(R, Ro, S):
    assert_residual_parity(R, Ro, S, rel=MIXED_ENTRY)
    norm = np.abs(R - Ro).reshape(-1, 5).max(axis=0) / np.abs(Ro).reshape(-1, 5).max(axis=0)
    assert np.all(norm <= MIXED_NORM), norm
    return norm


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_mixed_residual_all_orders(p):
    n = 4 if p <= 4 else 3
    d = I.hex_box_mesh((n, n, n), seed=p, shuffle=True, rotate=True, perturb=0.1)
    phys = I.tgv_physics(Ma=0.2, Re=200.0)
    ora = HexFR(d, phys, p)
    Q = np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.2, perturb=1e-2, seed=p))
    with fr.Mesh(d, _mixed(phys), p) as g:
        g.set_state(Q)
        _check(g.residual(), ora.residual(Q), ora.residual(Q, magnitude=True))


def test_mixed_residual_tgv_ma01_8cube_p3():
    d = I.hex_box_mesh((8, 8, 8), seed=0, shuffle=True, rotate=True)
    phys = I.tgv_physics()
    ora = HexFR(d, phys, 3)
    Q = np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.1, perturb=1e-3))
    with fr.Mesh(d, _mixed(phys), 3) as g:
        g.set_state(Q)
        _check(g.residual(), ora.residual(Q), ora.residual(Q, magnitude=True))


def test_mixed_rk44_steps():
    d = I.hex_box_mesh((4, 4, 4), seed=2, rotate=True, shuffle=True)
    phys = I.tgv_physics()
    ora = HexFR(d, phys, 3)
    Q = np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.1))
    dt = ora.max_dt(Q, 0.3)
    with fr.Mesh(d, _mixed(phys), 3) as g:
        g.set_state(Q)
        Qo, t = Q.copy(), 0.0
        for _ in range(5):
            g.rk_step(t, dt)
            Qo = ora.rk44_step(Qo, t, dt)
            t += dt
        assert_state_parity(g.get_state(), Qo, ora.residual(Q, magnitude=True), t, rel=MIXED_ENTRY)


@pytest.mark.parametrize("kinds", [
    ((I.BC_WALL_ISOTHERMAL, (1.1,)), (I.BC_CHAR_OUTFLOW, (0.7,))),
    ((I.BC_CHAR_INFLOW, (0.9, 1.05, 1.0, 0.2, 0.0)), (I.BC_DIRICHLET, (1.0, 0.1, 0.0, 0.0, 1.8)))])
def test_mixed_boundary_conditions(kinds):
    d = I.hex_box_mesh((3, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, True),
                       wall_tags={1: kinds[0], 2: kinds[1]}, seed=3, rotate=True, perturb=0.1)
    phys = I.Physics(gamma=1.4, R=1.0, mu=0.02, Pr=0.71, viscous=1)

    def st(X):
        return I.conserved(1 + 0.1 * np.sin(X[..., 0]), 0.2 * np.cos(X[..., 1] * 2 * np.pi),
                           0.1 + 0 * X[..., 0], 0.05 * np.sin(2 * np.pi * X[..., 2]), 0.7 + 0.02 * X[..., 0], 1.4)
    ora = HexFR(d, phys, 3)
    Q = np.ascontiguousarray(st(ora.x))
    with fr.Mesh(d, _mixed(phys), 3) as g:
        g.set_state(Q)
        _check(g.residual(), ora.residual(Q), ora.residual(Q, magnitude=True))


def test_mixed_euler_free_stream():
    d = I.hex_box_mesh((3, 3, 2), seed=5, rotate=True, perturb=0.15)
    phys = I.Physics(gamma=1.4, R=1.0, mu=0.0, viscous=0, precision=1)
    ora = HexFR(d, phys, 4)
    U = np.ascontiguousarray(I.uniform_state(ora.x.shape[:2]))
    with fr.Mesh(d, phys, 4) as g:
        g.set_state(U)
        R = g.residual()
    # double-float arithmetic: uniform flow stays steady to ~2^-44 of the flux scale
    assert np.abs(R).max() <= 1e-11 * 1.5 / ora.h.min()
