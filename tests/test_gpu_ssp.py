"""SSP Runge-Kutta stages (FR_SSPRK33, FR_SSPRK104) on the GPU vs the oracle's integrators
(marked gpu): two steps on a hexahedral and on a mixed hexahedral/prismatic mesh, both precisions;
states within 1e-12 (FP64) / 1e-9 (mixed) of (|Q| + t S)."""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle import timeint as TI
from oracle.mixedfr import MixedFR

from helpers import assert_state_parity, ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


@pytest.mark.parametrize("scheme,name", [(fr.FR_SSPRK33, "ssprk33"), (fr.FR_SSPRK104, "ssprk104")])
@pytest.mark.parametrize("prisms", [None, "checker"])
@pytest.mark.parametrize("precision,rel", [(0, 1e-12), (1, 1e-9)])
def test_ssp_steps(scheme, name, prisms, precision, rel):
    p = 3
    d = I.hex_box_mesh((3, 3, 2), prisms=prisms, seed=5, rotate=True, shuffle=True, perturb=0.05)
    ph = I.tgv_physics(Ma=0.2, Re=300.0)
    ora = MixedFR(d, ph, p)
    Qs = [np.ascontiguousarray(I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=2)) for x in ora.x]
    dt = 2e-3 if scheme == fr.FR_SSPRK33 else 6e-3
    ph.precision = precision
    with fr.Mesh(d, ph, p) as g:
        g.set_state(np.ascontiguousarray(np.concatenate([q.reshape(-1, 5) for q in Qs])))
        for k in range(2):
            g.rk_step(k * dt, dt, scheme)
        Qg = g.get_state().reshape(-1, 5)
    Q = Qs
    for _ in range(2):
        Q = TI.SCHEMES[name](ora.residual, Q, dt)
    S = np.concatenate([s.reshape(-1, 5) for s in ora.residual(Qs, magnitude=True)])
    assert_state_parity(Qg, np.concatenate([q.reshape(-1, 5) for q in Q]), S, 2 * dt * TI.STAGES[name] / 4, rel=rel)


def test_unknown_scheme_and_stage_rejected():
    d = I.hex_box_mesh((2, 2, 2))
    with fr.Mesh(d, I.tgv_physics(), 2) as g:
        g.set_state(np.ascontiguousarray(I.uniform_state((g.n_elem, g.n_pts))))
        with pytest.raises(fr.FRError, match="FR_EINVAL"):
            g.rk_stage(0, 0.0, 1e-3, scheme=7)
        with pytest.raises(fr.FRError, match="FR_EINVAL"):
            g.rk_stage(3, 0.0, 1e-3, scheme=fr.FR_SSPRK33)
