"""Tensor-core face interpolation (FR_PREC_MIXED_TC) vs the FP64 oracle, through the C ABI.

The solution traces are contracted by tcgen05.mma on exponent-aligned TF32 slices (error-free
splitting), the rest of the residual as in FR_PREC_MIXED.  Same error bars as the double-float
path: per entry |R - R_oracle| <= 1e-9 S, normwise <= 1e-6 per variable; the per-variable
errors are printed (run with -s).  The residual is also compared with FR_PREC_MIXED's (the only
difference is the interpolation's arithmetic).
"""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle.hexfr import HexFR

from helpers import assert_residual_parity, assert_state_parity, ensure_lib

pytestmark = pytest.mark.gpu

ENTRY, NORM = 1e-9, 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _prec(phys, precision):
    ph = I.Physics(**{k: getattr(phys, k) for k in phys.__dataclass_fields__})
    ph.precision = precision
    return ph


def _errors(R, Ro, S):
    entry = (np.abs(R - Ro) / S).reshape(-1, 5).max(axis=0)
    norm = np.abs(R - Ro).reshape(-1, 5).max(axis=0) / np.abs(Ro).reshape(-1, 5).max(axis=0)
    return entry, norm


@pytest.mark.parametrize("Ma", [0.1, 0.3])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_tc_residual_against_oracle(p, Ma):
    n = 4 if p <= 4 else 3
    d = I.hex_box_mesh((n, n, n), seed=p, shuffle=True, rotate=True, perturb=0.1)
    phys = I.tgv_physics(Ma=Ma, Re=400.0)
    ora = HexFR(d, phys, p)
    Q = np.ascontiguousarray(I.tgv_state(ora.x, Ma=Ma, perturb=1e-2, seed=p))
    Ro, S = ora.residual(Q), ora.residual(Q, magnitude=True)
    with fr.Mesh(d, _prec(phys, fr.FR_PREC_MIXED_TC), p) as g, fr.Mesh(d, _prec(phys, 1), p) as m:
        g.set_state(Q)
        m.set_state(Q)
        R, Rm = g.residual(), m.residual()
    entry, norm = _errors(R, Ro, S)
    print(f"p={p} Ma={Ma}: tensor-core traces, per-entry error / S {entry}, normwise {norm}")
    assert_residual_parity(R, Ro, S, rel=ENTRY)
    assert np.all(norm <= NORM), norm
    assert_residual_parity(R, Rm, S, rel=ENTRY)


def test_tc_boundaries_and_rk44_steps():
    d = I.hex_box_mesh((3, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, True),
                       wall_tags={1: (I.BC_WALL_ISOTHERMAL, (1.1,)), 2: (I.BC_CHAR_OUTFLOW, (0.7,))},
                       seed=3, rotate=True, shuffle=True, perturb=0.1)
    phys = I.Physics(gamma=1.4, R=1.0, mu=0.02, Pr=0.71, viscous=1)
    p = 3
    ora = HexFR(d, phys, p)
    Q = np.ascontiguousarray(I.conserved(1 + 0.1 * np.sin(ora.x[..., 0]), 0.2 * np.cos(ora.x[..., 1] * 2 * np.pi),
                                         0.1 + 0 * ora.x[..., 0], 0.05 * np.sin(2 * np.pi * ora.x[..., 2]),
                                         0.7 + 0.02 * ora.x[..., 0], 1.4))
    S = ora.residual(Q, magnitude=True)
    with fr.Mesh(d, _prec(phys, fr.FR_PREC_MIXED_TC), p) as g:
        g.set_state(Q)
        assert_residual_parity(g.residual(), ora.residual(Q), S, rel=ENTRY)
        dt = 0.3 * ora.max_dt(Q, 0.3)
        Qo, t = Q.copy(), 0.0
        for _ in range(3):
            g.rk_step(t, dt)                   # no FR_ETIMEOUT / FR_ENONFINITE from the flag word
            Qo = ora.rk44_step(Qo, t, dt)
            t += dt
        assert_state_parity(g.get_state(), Qo, S, t, rel=ENTRY)


def test_tc_not_batched():
    d = I.hex_box_mesh((2, 2, 2))
    with fr.Mesh(d, _prec(I.tgv_physics(), fr.FR_PREC_MIXED_TC), 2) as g:
        with pytest.raises(fr.FRError) as ei:
            fr.Batch([g])
        assert ei.value.status == fr.FR_EUNSUPPORTED


def test_tc_unperturbed_low_mach_tgv_normwise():
    """The benchmark's state (unperturbed TGV, Ma 0.1, Re 1600) at p = 4: its continuity residual
    is small, so trace errors amplified by the Rusanov dissipation show most here (with four
    slices the error reached 1e-6 of the largest entry)."""
    d = I.hex_box_mesh((10, 10, 10))
    phys = I.tgv_physics()
    p = 4
    ora = HexFR(d, phys, p)
    Q = np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.1))
    Ro, S = ora.residual(Q), ora.residual(Q, magnitude=True)
    with fr.Mesh(d, _prec(phys, fr.FR_PREC_MIXED_TC), p) as g:
        g.set_state(Q)
        R = g.residual()
    entry, norm = _errors(R, Ro, S)
    print(f"unperturbed TGV p=4: per-entry error / S {entry}, normwise {norm}")
    assert np.all(norm <= 1e-7), norm
    # In this symmetric state the fluxes and jumps vanish at some points, where the magnitude
    # scale S goes to zero although the Rusanov dissipation still rounds at the size of the
    # traces themselves: the per-entry bar takes a floor of 1e-3 of each variable's largest S.
    Sf = np.maximum(S.reshape(-1, 5), 1e-3 * S.reshape(-1, 5).max(axis=0)).reshape(S.shape)
    assert_residual_parity(R, Ro, Sf, rel=ENTRY)
