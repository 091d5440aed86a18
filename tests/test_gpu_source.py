"""Source term S (body force, sponge) on the GPU vs the oracle (marked gpu): residuals of a hexahedral
and a mixed mesh in both precisions, an RK step, and switching parts off."""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle import timeint as TI
from oracle.mixedfr import MixedFR

from helpers import assert_residual_parity, assert_state_parity, ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def flat(arrs):
    return np.concatenate([np.asarray(a).reshape(-1, 5) for a in arrs])


@pytest.mark.parametrize("prisms", [None, "checker"])
@pytest.mark.parametrize("precision,rel", [(0, 1e-12), (1, 1e-9)])
def test_source_residual_and_step(prisms, precision, rel):
    d = I.hex_box_mesh((3, 3, 2), prisms=prisms, seed=3, rotate=True, shuffle=True, perturb=0.1)
    ph = I.tgv_physics(Ma=0.2, Re=300.0)
    ora = MixedFR(d, ph, 3)
    Qs = [np.ascontiguousarray(I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=3)) for x in ora.x]
    g = (0.3, -0.2, 0.1)
    sig = [2.0 * (0.5 + 0.5 * np.tanh(x[..., 0] - np.pi)) for x in ora.x]
    ref = [I.uniform_state(x.shape[:2], rho=1.0, vel=(1.0, 0.0, 0.0), p=1 / (1.4 * 0.04)) for x in ora.x]
    ora.set_source(accel=g, sigma=sig, Q_ref=ref)
    ph.precision = precision
    with fr.Mesh(d, ph, 3) as m:
        m.set_state(flat(Qs))
        m.set_source(accel=g, sigma=np.concatenate([s.ravel() for s in sig]), Q_ref=flat(ref))
        R = m.residual()
        assert_residual_parity(R.reshape(-1, 5), flat(ora.residual(Qs)), flat(ora.residual(Qs, magnitude=True)),
                               rel=rel)
        dt = 2e-3
        m.rk_step(0.0, dt)
        want = TI.rk44(ora.residual, Qs, dt)
        assert_state_parity(m.get_state().reshape(-1, 5), flat(want), flat(ora.residual(Qs, magnitude=True)), dt,
                            rel=rel)
        # switching everything off restores the plain residual
        m.set_state(flat(Qs))
        m.set_source()
        ora.set_source()
        assert_residual_parity(m.residual().reshape(-1, 5), flat(ora.residual(Qs)),
                               flat(ora.residual(Qs, magnitude=True)), rel=rel)
