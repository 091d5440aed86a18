"""Order projection (fr_project_state) on the GPU vs the oracle (marked gpu): up and down between
orders on hexahedral, mixed and curved meshes; the projected state then steps."""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle import project as PJ
from oracle.mixedfr import MixedFR

from helpers import ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def flat(arrs):
    return np.concatenate([np.asarray(a).reshape(-1, 5) for a in arrs])


@pytest.mark.parametrize("p,q", [(1, 3), (2, 5), (5, 3), (7, 2), (4, 4)])
@pytest.mark.parametrize("kind", ["hex", "mixed", "curved"])
def test_projection(p, q, kind):
    if kind == "curved":
        d = I.curved_box_mesh((2, 2, 2), prisms="checker", warp=0.1, seed=2, rotate=True, shuffle=True)
    else:
        d = I.hex_box_mesh((3, 3, 2), prisms=None if kind == "hex" else "checker", seed=2, rotate=True, shuffle=True,
                           perturb=0.1)
    ph = I.tgv_physics(Ma=0.2, Re=300.0)
    ora = MixedFR(d, ph, p)
    Qs = [np.ascontiguousarray(I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=3)) for x in ora.x]
    want = flat(PJ.project(Qs, p, q))
    with fr.Mesh(d, ph, p) as a, fr.Mesh(d, ph, q) as b:
        a.set_state(flat(Qs))
        fr.project_state(a, b)
        got = b.get_state().reshape(-1, 5)
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13 * np.abs(want).max())
        b.rk_step(0.0, 1e-3)
        assert np.isfinite(b.get_state()).all()


def test_projection_rejects_different_meshes():
    ph = I.tgv_physics()
    with fr.Mesh(I.hex_box_mesh((2, 2, 2)), ph, 2) as a, fr.Mesh(I.hex_box_mesh((3, 2, 2)), ph, 2) as b:
        a.set_state(np.ascontiguousarray(I.uniform_state((a.n_elem, a.n_pts))))
        with pytest.raises(fr.FRError, match="FR_EINVAL"):
            fr.project_state(a, b)
