"""fr_residual_static: the residual computed with the library's static scratch array.

For callers that cannot allocate device memory when they need a residual (the entry point
allocates nothing; its intermediates live in a fixed 32 MiB device array).  Its output must agree
with fr_residual on the same state, within the residual bar the other tests use, on two calls
in a row (the second call sees the first call's leftovers in the shared array).  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle.hexfr import HexFR

from helpers import assert_residual_parity, ensure_lib

pytestmark = pytest.mark.gpu


def test_static_scratch_residual_matches_fr_residual_twice():
    torch = pytest.importorskip("torch")
    ensure_lib()
    d = I.hex_box_mesh((8, 8, 8), seed=0, shuffle=True, rotate=True, perturb=0.05)
    phys = I.tgv_physics()
    ora = HexFR(d, phys, 3)
    with fr.Mesh(d, phys, 3) as g:
        for seed in (1, 2):
            Q = np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.1, perturb=1e-3, seed=seed))
            Qd = torch.from_numpy(Q).cuda()
            g.set_state(Qd)
            R_ref = torch.empty_like(Qd)
            g.residual(out=R_ref)
            R_new = torch.full_like(Qd, float("nan"))
            g.residual_static(Qd, R_new)
            torch.cuda.synchronize()
            S = ora.residual(Q, magnitude=True)
            assert_residual_parity(R_new.cpu().numpy(), R_ref.cpu().numpy(), S)


def test_static_scratch_rejects_oversized_mesh():
    torch = pytest.importorskip("torch")
    ensure_lib()
    d = I.hex_box_mesh((24, 24, 24))
    with fr.Mesh(d, I.tgv_physics(), 4) as g:
        Qd = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        R = torch.zeros_like(Qd)
        with pytest.raises(fr.FRError) as ei:
            g.residual_static(Qd, R)
        assert ei.value.status == fr.FR_EINVAL
        assert "static array holds" in str(ei.value)
