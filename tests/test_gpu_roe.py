"""Roe common flux on the GPU vs the oracle (marked gpu): hexahedral and mixed meshes, boundary
conditions, both precisions.  Bars as for Rusanov: per entry <= 1e-12 S (FP64) / 1e-9 S (mixed)."""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle.hexfr import HexFR
from oracle.mixedfr import MixedFR

from helpers import assert_residual_parity, ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _roe(ph, precision=0):
    ph.inviscid_flux = 1
    ph.precision = precision
    return ph


@pytest.mark.parametrize("p,precision", [(2, 0), (4, 0), (3, 1), (5, 1)])
def test_roe_tgv_hex(p, precision):
    d = I.hex_box_mesh((3, 3, 3), seed=p, rotate=True, shuffle=True, perturb=0.1)
    ph = _roe(I.tgv_physics(Ma=0.3, Re=300.0), precision)
    ora = HexFR(d, ph, p)
    Q = np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.3, perturb=2e-2, seed=p))
    with fr.Mesh(d, ph, p) as g:
        g.set_state(Q)
        R = g.residual()
    assert_residual_parity(R, ora.residual(Q), ora.residual(Q, magnitude=True), rel=1e-12 if precision == 0 else 1e-9)


def test_roe_walls_and_characteristic_boundaries():
    d = I.hex_box_mesh((3, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, False), seed=3, rotate=True, perturb=0.1,
                       wall_tags={1: (I.BC_CHAR_INFLOW, (0.9, 1.05, 1.0, 0.2, 0.0)), 2: (I.BC_CHAR_OUTFLOW, (0.7,)),
                                  5: (I.BC_WALL_ISOTHERMAL, (1.1,)), 6: (I.BC_WALL_ISOTHERMAL, (0.9,))})
    ph = _roe(I.Physics(gamma=1.4, R=1.0, mu=0.02, Pr=0.71, viscous=1))

    def st(X):
        return I.conserved(1 + 0.1 * np.sin(X[..., 0]), 0.3 + 0.1 * np.cos(2 * np.pi * X[..., 1]), 0.05 + 0 * X[..., 0],
                           0.02 * np.sin(2 * np.pi * X[..., 2]), 0.7 + 0.02 * X[..., 0], 1.4)
    ora = HexFR(d, ph, 3)
    Q = np.ascontiguousarray(st(ora.x))
    with fr.Mesh(d, ph, 3) as g:
        g.set_state(Q)
        R = g.residual()
    assert_residual_parity(R, ora.residual(Q), ora.residual(Q, magnitude=True), rel=1e-12)


def test_roe_mixed_mesh():
    d = I.hex_box_mesh((3, 3, 2), prisms="checker", seed=6, rotate=True, shuffle=True, perturb=0.1)
    ph = _roe(I.tgv_physics(Ma=0.3, Re=300.0))
    ora = MixedFR(d, ph, 3)
    Qs = [np.ascontiguousarray(I.tgv_state(x, Ma=0.3, perturb=2e-2, seed=6)) for x in ora.x]
    flat = lambda a: np.concatenate([b.reshape(-1, 5) for b in a])  # noqa: E731
    with fr.Mesh(d, ph, 3) as g:
        g.set_state(flat(Qs))
        R = g.residual()
    assert_residual_parity(R, flat(ora.residual(Qs)), flat(ora.residual(Qs, magnitude=True)), rel=1e-12)
