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


def test_static_scratch_large_then_small_mesh_with_boundaries():
    """A larger periodic mesh at p = 3, then a smaller walled mesh at p = 2 with characteristic
    outflow: the second call finds the first call's larger layout in the shared array and must
    still match fr_residual."""
    torch = pytest.importorskip("torch")
    ensure_lib()
    d1 = I.hex_box_mesh((8, 8, 8), seed=4, shuffle=True, rotate=True, perturb=0.05)
    phys1 = I.tgv_physics()
    d2 = I.hex_box_mesh((3, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, True),
                        wall_tags={1: (I.BC_WALL_ISOTHERMAL, (1.1,)), 2: (I.BC_CHAR_OUTFLOW, (0.7,))},
                        seed=3, rotate=True, shuffle=True, perturb=0.1)
    phys2 = I.Physics(gamma=1.4, R=1.0, mu=0.02, Pr=0.71, viscous=1)

    def st2(X):
        return I.conserved(1 + 0.1 * np.sin(X[..., 0]), 0.2 * np.cos(X[..., 1] * 2 * np.pi),
                           0.1 + 0 * X[..., 0], 0.05 * np.sin(2 * np.pi * X[..., 2]), 0.7 + 0.02 * X[..., 0], 1.4)

    for d, phys, p, state in ((d1, phys1, 3, lambda x: I.tgv_state(x, Ma=0.1, perturb=1e-3, seed=5)),
                              (d2, phys2, 2, st2)):
        ora = HexFR(d, phys, p)
        Q = np.ascontiguousarray(state(ora.x))
        with fr.Mesh(d, phys, p) as g:
            Qd = torch.from_numpy(Q).cuda()
            g.set_state(Qd)
            R_ref = torch.empty_like(Qd)
            g.residual(out=R_ref)
            R_new = torch.full_like(Qd, float("nan"))
            g.residual_static(Qd, R_new)
            torch.cuda.synchronize()
            assert_residual_parity(R_new.cpu().numpy(), R_ref.cpu().numpy(), ora.residual(Q, magnitude=True))


def test_static_scratch_refusals_leave_the_mesh_usable():
    """Each documented refusal is FR_EUNSUPPORTED (double-float meshes, prisms, c != 0, the
    eddy-viscosity closure); wrong
    tensor sizes are refused by the binding before the library is called.  A refused call does
    not poison the mesh."""
    torch = pytest.importorskip("torch")
    ensure_lib()
    d = I.hex_box_mesh((2, 2, 2))
    cases = [(d, I.Physics(gamma=1.4, R=1.0, mu=0.01, Pr=0.71, viscous=1, precision=1), "FP64 meshes only"),
             (I.hex_box_mesh((2, 2, 2), prisms="all"), I.tgv_physics(), "hexahedral meshes only"),
             (d, I.Physics(gamma=1.4, R=1.0, mu=0.01, Pr=0.71, viscous=1, vcjh_c=0.01), "c = 0")]
    cases.append((d, I.tgv_physics(), "closure"))
    for desc, phys, msg in cases:
        with fr.Mesh(desc, phys, 2) as g:
            if msg == "closure":
                g.set_closure(np.zeros(9153, np.float32), np.r_[np.zeros(11), np.ones(11), 1.0])
            Qd = torch.from_numpy(np.ascontiguousarray(I.uniform_state(g.shape[:-1]))).cuda()
            g.set_state(Qd)
            R = torch.zeros_like(Qd)
            with pytest.raises(fr.FRError) as ei:
                g.residual_static(Qd, R)
            assert ei.value.status == fr.FR_EUNSUPPORTED and msg in str(ei.value)
            g.residual()     # still usable
    with fr.Mesh(d, I.tgv_physics(), 2) as g:
        Qd = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        with pytest.raises(ValueError):
            g.residual_static(Qd, torch.zeros(Qd.numel() - 5, dtype=torch.float64, device="cuda"))
        g.set_state(Qd + 1.0)
        g.residual()
