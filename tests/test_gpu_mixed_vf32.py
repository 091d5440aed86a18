"""Double-float path with the viscous branch in FP32 (FR_PREC_MIXED_VF32) vs the FP64 oracle.

The viscous branch (corrected gradients of the perturbation from each element's first point,
gradient traces, stress and heat flux, the interface viscous flux) runs in FP32; its rounding is
about 1e-6 of the viscous part of the residual, so relative to the residual it grows like 1/Re
and with the viscous share.  Asserted on perturbed TGV states for Re >= 400 (Ma <= 0.5, p <= 7):
  per entry   |R - R_oracle| <= 2e-8 * S
  normwise    max|R - R_oracle| / max|R_oracle| <= 1e-6 per variable.
(States whose residual is almost purely viscous, like the initial TGV state of the benchmark,
exceed the normwise figure: 2.1e-6 there.)  The errors are printed per variable (run with -s); a
low-Re case documents the growth."""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle.hexfr import HexFR

from helpers import assert_residual_parity, assert_state_parity, ensure_lib

pytestmark = pytest.mark.gpu

ENTRY, NORM = 2e-8, 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _vf32(phys):
    ph = I.Physics(**{k: getattr(phys, k) for k in phys.__dataclass_fields__})
    ph.precision = fr.FR_PREC_MIXED_VF32
    return ph


def _errors(R, Ro, S):
    entry = (np.abs(R - Ro) / S).reshape(-1, 5).max(axis=0)
    norm = np.abs(R - Ro).reshape(-1, 5).max(axis=0) / np.abs(Ro).reshape(-1, 5).max(axis=0)
    return entry, norm


def _case(p, Ma, Re, seed):
    n = 4 if p <= 4 else 3
    d = I.hex_box_mesh((n, n, n), seed=seed, shuffle=True, rotate=True, perturb=0.1)
    phys = I.tgv_physics(Ma=Ma, Re=Re)
    ora = HexFR(d, phys, p)
    Q = np.ascontiguousarray(I.tgv_state(ora.x, Ma=Ma, perturb=1e-2, seed=seed))
    with fr.Mesh(d, _vf32(phys), p) as g:
        g.set_state(Q)
        R = g.residual()
    return R, ora.residual(Q), ora.residual(Q, magnitude=True)


@pytest.mark.parametrize("Re", [400.0, 1600.0])
@pytest.mark.parametrize("Ma", [0.1, 0.5])
@pytest.mark.parametrize("p", [1, 3, 5, 7])
def test_vf32_residual_within_stated_error(p, Ma, Re):
    R, Ro, S = _case(p, Ma, Re, seed=p)
    entry, norm = _errors(R, Ro, S)
    print(f"p={p} Ma={Ma} Re={Re}: per-entry error / S {entry.max():.2e}, normwise {norm.max():.2e}")
    assert_residual_parity(R, Ro, S, rel=ENTRY)
    assert np.all(norm <= NORM), norm


def test_vf32_error_grows_like_inverse_reynolds():
    """The FP32 branch is scaled by the viscosity: a 16x smaller Re gives a larger error (documents
    why the stated error holds from Re = 400 up)."""
    e_hi = _errors(*_case(4, 0.3, 1600.0, 4))[1].max()
    e_lo = _errors(*_case(4, 0.3, 100.0, 4))[1].max()
    assert e_lo > 4 * e_hi, (e_lo, e_hi)


def test_vf32_walls_and_rk44_steps():
    d = I.hex_box_mesh((3, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, True),
                       wall_tags={1: (I.BC_WALL_ISOTHERMAL, (1.1,)), 2: (I.BC_CHAR_OUTFLOW, (0.7,))},
                       seed=3, rotate=True, shuffle=True, perturb=0.1)
    phys = I.Physics(gamma=1.4, R=1.0, mu=5e-4, Pr=0.71, viscous=1)       # Re = rho |u| L / mu ~ 400
    p = 3
    ora = HexFR(d, phys, p)
    Q = np.ascontiguousarray(I.conserved(1 + 0.1 * np.sin(ora.x[..., 0]), 0.2 * np.cos(ora.x[..., 1] * 2 * np.pi),
                                         0.1 + 0 * ora.x[..., 0], 0.05 * np.sin(2 * np.pi * ora.x[..., 2]),
                                         0.7 + 0.02 * ora.x[..., 0], 1.4))
    S = ora.residual(Q, magnitude=True)
    with fr.Mesh(d, _vf32(phys), p) as g:
        g.set_state(Q)
        assert_residual_parity(g.residual(), ora.residual(Q), S, rel=ENTRY)
        dt = 0.3 * ora.max_dt(Q, 0.3)
        Qo, t = Q.copy(), 0.0
        for _ in range(3):
            g.rk_step(t, dt)
            Qo = ora.rk44_step(Qo, t, dt)
            t += dt
        assert_state_parity(g.get_state(), Qo, S, t, rel=ENTRY)


def test_vf32_refusals():
    d = I.hex_box_mesh((2, 2, 2))
    phys = _vf32(I.tgv_physics())
    phys.vcjh_c = 0.01
    with pytest.raises(fr.FRError) as ei:
        fr.Mesh(d, phys, 2)
    assert ei.value.status == fr.FR_EUNSUPPORTED
    with fr.Mesh(d, _vf32(I.tgv_physics()), 2) as g:
        with pytest.raises(fr.FRError) as ei:
            fr.Batch([g])
        assert ei.value.status == fr.FR_EUNSUPPORTED
