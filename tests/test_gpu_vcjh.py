"""Correction functions c != 0 of the energy-stable family on the GPU vs the oracles (marked gpu).

Hexahedral meshes (straight and curved), BR2 and LDG, Rusanov and Roe, walls and characteristic
boundaries, both precisions; per entry <= 1e-12 S (FP64) / <= 1e-9 S (double-float), RK44 states
within 1e-12 (|Q| + t S).  The kernels that read the mesh's own tables give bit-identical results
to the constant-memory ones when c is so small that the tables coincide.  Unsupported
combinations (prisms, batches, the allocation-free entry point) and c outside the family are
refused.
"""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle.hexfr import HexFR
from oracle.mixedfr import MixedFR

from helpers import assert_residual_parity, assert_state_parity, ensure_lib, vcjh_c

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _tgv(c, precision=0, viscous=1):
    ph = I.tgv_physics(Ma=0.2, Re=300.0)
    ph.vcjh_c, ph.precision, ph.viscous = c, precision, viscous
    return ph


CASES = [(1, "sd"), (2, "hu"), (3, "neg"), (4, "sd"), (5, "big"), (7, "hu")]


@pytest.mark.parametrize("p,which", CASES)
@pytest.mark.parametrize("precision,rel", [(0, 1e-12), (1, 1e-9)])
def test_vcjh_hex_residual(p, which, precision, rel):
    c = vcjh_c(p, which)
    d = I.hex_box_mesh((3, 3, 2) if p < 6 else (2, 2, 2), seed=30 + p, rotate=True, shuffle=True, perturb=0.1)
    ora = HexFR(d, _tgv(c), p)
    Q = np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.2, perturb=1e-2, seed=p))
    with fr.Mesh(d, _tgv(c, precision), p) as g:
        g.set_state(Q)
        R = g.residual()
    assert_residual_parity(R, ora.residual(Q), ora.residual(Q, magnitude=True), rel=rel)


@pytest.mark.parametrize("viscous", [1, 2])
def test_vcjh_roe_walls_and_characteristic_boundaries(viscous):
    d = I.hex_box_mesh((3, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, True), seed=3, rotate=True, perturb=0.1,
                       wall_tags={1: (I.BC_CHAR_INFLOW, (0.9, 1.05, 1.0, 0.2, 0.0)), 2: (I.BC_WALL_ISOTHERMAL, (1.1,))})
    p = 3
    ph = I.Physics(gamma=1.4, R=1.0, mu=0.02, Pr=0.71, viscous=viscous, inviscid_flux=1, vcjh_c=vcjh_c(p, "sd"))
    ora = HexFR(d, ph, p)
    X = ora.x
    Q = np.ascontiguousarray(I.conserved(1 + 0.1 * np.sin(X[..., 0]), 0.2 + 0.1 * np.cos(X[..., 1]), 0.1 + 0 * X[..., 0],
                                         0.05 * np.sin(2 * X[..., 2]), 0.7 + 0.02 * X[..., 0], 1.4))
    for precision, rel in ((0, 1e-12), (1, 1e-9)):
        ph.precision = precision
        with fr.Mesh(d, ph, p) as g:
            g.set_state(Q)
            R = g.residual()
        assert_residual_parity(R, ora.residual(Q), ora.residual(Q, magnitude=True), rel=rel)


def test_vcjh_curved_mesh():
    d = I.curved_box_mesh((2, 2, 2), warp=0.12, seed=5, rotate=True, shuffle=True)
    p = 4
    c = vcjh_c(p, "hu")
    ora = MixedFR(d, _tgv(c), p)
    Qs = [np.ascontiguousarray(I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=5)) for x in ora.x]
    for precision, rel in ((0, 1e-12), (1, 1e-9)):
        with fr.Mesh(d, _tgv(c, precision), p) as g:
            g.set_state(Qs[0])
            R = g.residual()
        assert_residual_parity(R, ora.residual(Qs)[0], ora.residual(Qs, magnitude=True)[0], rel=rel)


@pytest.mark.parametrize("precision,rel", [(0, 1e-12), (1, 1e-9)])
def test_vcjh_rk44_steps(precision, rel):
    d = I.hex_box_mesh((3, 3, 2), seed=9, rotate=True, shuffle=True, perturb=0.1)
    p = 3
    c = vcjh_c(p, "hu")
    ora = HexFR(d, _tgv(c), p)
    Q0 = np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.2, perturb=1e-2, seed=9))
    dt = 0.5 * ora.max_dt(Q0, 0.3)
    Q = Q0
    for s in range(3):
        Q = ora.rk44_step(Q, s * dt, dt)
    with fr.Mesh(d, _tgv(c, precision), p) as g:
        g.set_state(Q0)
        for s in range(3):
            g.rk_step(s * dt, dt)
        Qg = g.get_state()
    assert_state_parity(Qg, Q, ora.residual(Q0, magnitude=True), 3 * dt, rel=rel)


@pytest.mark.parametrize("precision", [0, 1])
def test_vcjh_tables_match_constant_path(precision):
    """c = 1e-300 leaves every table entry unchanged, so the kernels on the mesh's own tables
    must reproduce the constant-memory kernels bit for bit."""
    d = I.hex_box_mesh((3, 3, 2), seed=12, rotate=True, shuffle=True, perturb=0.1)
    p = 4
    x = None
    out = []
    for c in (0.0, 1e-300):
        with fr.Mesh(d, _tgv(c, precision), p) as g:
            if x is None:
                x = g.solution_points()
            g.set_state(np.ascontiguousarray(I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=12)))
            out.append(g.residual())
    assert np.array_equal(out[0], out[1])


def test_vcjh_refusals():
    torch = pytest.importorskip("torch")
    p = 3
    c = vcjh_c(p, "sd")
    with pytest.raises(fr.FRError, match="FR_EUNSUPPORTED"):
        fr.Mesh(I.hex_box_mesh((2, 2, 2), prisms="checker", seed=1), _tgv(c), p)
    c_minus = 2.0 * vcjh_c(p, "neg")
    for bad in (c_minus * (1 + 1e-9), 2.0 * c_minus, float("nan"), float("inf")):
        with pytest.raises(fr.FRError, match="FR_EINVAL"):
            fr.Mesh(I.hex_box_mesh((2, 2, 2), seed=1), _tgv(bad), p)
    d = I.hex_box_mesh((2, 2, 2), seed=2)
    with fr.Mesh(d, _tgv(c), p) as g:
        with pytest.raises(fr.FRError, match="FR_EUNSUPPORTED"):
            fr.Batch([g])
        Q = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        with pytest.raises(fr.FRError, match="FR_EUNSUPPORTED"):
            g.residual_static(Q, torch.empty_like(Q))
