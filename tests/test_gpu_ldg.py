"""LDG viscous discretisation (FR_VISC_LDG) on the GPU vs the oracles (marked gpu): hexahedral,
mixed and curved meshes, walls and characteristic boundaries, both precisions, an RK step and
a batch; per entry <= 1e-12 S (FP64) / 1e-9 S (mixed)."""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle.hexfr import HexFR
from oracle.mixedfr import MixedFR

from helpers import assert_residual_parity, assert_state_parity, ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def flat(arrs):
    return np.concatenate([np.asarray(a).reshape(-1, 5) for a in arrs])


def _ldg(ph, precision=0, tau=0.1):
    ph.viscous, ph.ldg_tau, ph.precision = 2, tau, precision
    return ph


@pytest.mark.parametrize("p", [1, 3, 5, 7])
@pytest.mark.parametrize("precision,rel", [(0, 1e-12), (1, 1e-9)])
def test_ldg_hex(p, precision, rel):
    d = I.hex_box_mesh((3, 3, 2) if p < 6 else (2, 2, 2), seed=p, rotate=True, shuffle=True, perturb=0.1)
    ora = HexFR(d, _ldg(I.tgv_physics(Ma=0.2, Re=300.0)), p)
    Q = np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.2, perturb=1e-2, seed=p))
    with fr.Mesh(d, _ldg(I.tgv_physics(Ma=0.2, Re=300.0), precision), p) as g:
        g.set_state(Q)
        R = g.residual()
    assert_residual_parity(R, ora.residual(Q), ora.residual(Q, magnitude=True), rel=rel)


def test_ldg_walls_and_characteristic_boundaries():
    d = I.hex_box_mesh((3, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, True), seed=3, rotate=True, perturb=0.1,
                       wall_tags={1: (I.BC_CHAR_INFLOW, (0.9, 1.05, 1.0, 0.2, 0.0)), 2: (I.BC_WALL_ISOTHERMAL, (1.1,))})
    ph = _ldg(I.Physics(gamma=1.4, R=1.0, mu=0.02, Pr=0.71, viscous=1))
    ora = HexFR(d, ph, 3)
    X = ora.x
    Q = np.ascontiguousarray(I.conserved(1 + 0.1 * np.sin(X[..., 0]), 0.2 + 0.1 * np.cos(X[..., 1]), 0.1 + 0 * X[..., 0],
                                         0.05 * np.sin(2 * X[..., 2]), 0.7 + 0.02 * X[..., 0], 1.4))
    with fr.Mesh(d, ph, 3) as g:
        g.set_state(Q)
        R = g.residual()
    assert_residual_parity(R, ora.residual(Q), ora.residual(Q, magnitude=True), rel=1e-12)


@pytest.mark.parametrize("curved", [False, True])
def test_ldg_mixed_and_curved_meshes(curved):
    d = (I.curved_box_mesh((2, 2, 2), prisms="checker", warp=0.12, seed=4, rotate=True, shuffle=True) if curved else
         I.hex_box_mesh((3, 3, 2), prisms="checker", seed=4, rotate=True, shuffle=True, perturb=0.1))
    p = 4
    ora = MixedFR(d, _ldg(I.tgv_physics(Ma=0.2, Re=300.0)), p)
    Qs = [np.ascontiguousarray(I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=4)) for x in ora.x]
    for precision, rel in ((0, 1e-12), (1, 1e-9)):
        with fr.Mesh(d, _ldg(I.tgv_physics(Ma=0.2, Re=300.0), precision), p) as g:
            g.set_state(flat(Qs))
            R = g.residual()
        assert_residual_parity(R.reshape(-1, 5), flat(ora.residual(Qs)), flat(ora.residual(Qs, magnitude=True)),
                               rel=rel)


def test_ldg_rk_step_and_batch():
    d = I.hex_box_mesh((3, 3, 3), seed=8, rotate=True, shuffle=True)
    ph = _ldg(I.tgv_physics(Ma=0.2, Re=300.0))
    ora = HexFR(d, ph, 3)
    Q = np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.2, perturb=1e-2, seed=8))
    dt = 0.5 * ora.max_dt(Q, 0.3)
    with fr.Mesh(d, ph, 3) as g, fr.Mesh(d, ph, 3) as gb:
        g.set_state(Q)
        g.rk_step(0.0, dt)
        gb.set_state(Q)
        with fr.Batch([gb]) as b:
            b.set_dt([dt])
            b.rk_step(0.0)
        want = ora.rk44_step(Q, 0.0, dt)
        S = ora.residual(Q, magnitude=True)
        assert_state_parity(g.get_state(), want, S, dt)
        assert_state_parity(gb.get_state(), want, S, dt)
