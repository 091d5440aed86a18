"""Domain-decomposed stages on one GPU: a mesh split into 2..4 parts (fr_mesh_create_part), each
stage run as three phases per part with the halo traces moved between the parts' buffers in
between (as ranks would exchange them), must give the residual and RK steps of the whole mesh.
The parts run the same kernels on the same per-element data, so the results agree bit for bit."""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr, inputs as I

from helpers import ensure_lib

pytestmark = pytest.mark.gpu


class Parts:
    """All parts of one partition on the current GPU with in-process halo exchange."""

    def __init__(self, desc, phys, p, n_parts):
        import torch
        self.torch = torch
        self.part = fr.partition(desc, p, n_parts)
        self.meshes = [fr.PartMesh(desc, phys, p, self.part, r) for r in range(n_parts)]
        self.halo = [m.halo() for m in self.meshes]
        Nf = (p + 1) ** 2
        n = [max(1, h["n_halo"]) * 15 * Nf for h in self.halo]
        self.send = [torch.zeros(k, dtype=torch.float64, device="cuda") for k in n]
        self.recv = [torch.zeros(k, dtype=torch.float64, device="cuda") for k in n]
        self.Nf = Nf

    def exchange(self, nv):
        self.torch.cuda.synchronize()
        w = nv * self.Nf
        for r, h in enumerate(self.halo):
            for k, q in enumerate(h["peers"]):
                hq = self.halo[q]
                kk = list(hq["peers"]).index(r)
                b, e = h["peer_begin"][k], h["peer_begin"][k + 1]
                bq = hq["peer_begin"][kk]
                self.recv[q][bq * w:(bq + e - b) * w].copy_(self.send[r][b * w:e * w])

    def stage(self, scheme=fr.FR_RESIDUAL_ONLY, stage=0, dt=0.0, R=None):
        for m, s in zip(self.meshes, self.send):
            m.phase(0, send=s)
        self.exchange(5)
        for m, s, rv in zip(self.meshes, self.send, self.recv):
            m.phase(1, recv=rv, send=s)
        self.exchange(15)
        for r, (m, rv) in enumerate(zip(self.meshes, self.recv)):
            m.phase(2, scheme, stage, 0.0, dt, recv=rv, R=None if R is None else R[r])

    def set_state(self, Q):
        for m, h in zip(self.meshes, self.halo):
            m.set_state(np.ascontiguousarray(Q[h["elem_global"]]))

    def gather(self, arrays, shape):
        out = np.empty(shape)
        for a, h in zip(arrays, self.halo):
            out[h["elem_global"]] = a
        return out

    def close(self):
        for m in self.meshes:
            m.close()


def _state(x, kind):
    if kind == "tgv":
        return I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=3)
    return I.conserved(1 + 0.1 * np.sin(x[..., 0]), 0.2 * np.cos(x[..., 1] * 2 * np.pi), 0.1 + 0 * x[..., 0],
                       0.05 * np.sin(2 * np.pi * x[..., 2]), 0.7 + 0.02 * x[..., 0], 1.4)


CASES = {
    "periodic": (lambda: I.hex_box_mesh((4, 4, 3), seed=2, shuffle=True, rotate=True, perturb=0.05),
                 lambda: I.tgv_physics(Ma=0.2, Re=400.0), "tgv"),
    "walls": (lambda: I.hex_box_mesh((4, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, True),
                                     wall_tags={1: (I.BC_WALL_ISOTHERMAL, (1.1,)), 2: (I.BC_CHAR_OUTFLOW, (0.7,))},
                                     seed=3, rotate=True, shuffle=True, perturb=0.1),
              lambda: I.Physics(gamma=1.4, R=1.0, mu=0.02, Pr=0.71, viscous=1), "wall"),
    "ldg": (lambda: I.hex_box_mesh((3, 3, 3), seed=4, shuffle=True, rotate=True),
            lambda: I.Physics(gamma=1.4, R=1.0, mu=0.01, Pr=0.71, viscous=2), "tgv"),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("n_parts", [2, 4])
@pytest.mark.parametrize("precision", [0, 1])
def test_partitioned_residual_equals_whole_mesh(case, n_parts, precision):
    torch = pytest.importorskip("torch")
    ensure_lib()
    mk_desc, mk_phys, kind = CASES[case]
    desc, phys, p = mk_desc(), mk_phys(), 3
    phys.precision = precision
    with fr.Mesh(desc, phys, p) as whole:
        Q = np.ascontiguousarray(_state(whole.solution_points(), kind))
        whole.set_state(Q)
        R_whole = whole.residual()
    parts = Parts(desc, phys, p, n_parts)
    try:
        assert all(h["n_halo"] > 0 for h in parts.halo)
        parts.set_state(Q)
        Rd = [torch.empty(m.shape, dtype=torch.float64, device="cuda") for m in parts.meshes]
        parts.stage(R=Rd)
        torch.cuda.synchronize()
        R_parts = parts.gather([r.cpu().numpy() for r in Rd], R_whole.shape)
        np.testing.assert_array_equal(R_parts, R_whole)
    finally:
        parts.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_partitioned_rk44_steps_equal_whole_mesh(precision):
    torch = pytest.importorskip("torch")
    ensure_lib()
    desc = I.hex_box_mesh((4, 4, 4), seed=6, shuffle=True, rotate=True, perturb=0.05)
    phys = I.tgv_physics(Ma=0.2, Re=400.0)
    phys.precision = precision
    p = 2
    whole = fr.Mesh(desc, phys, p)
    Q = np.ascontiguousarray(I.tgv_state(whole.solution_points(), Ma=0.2, perturb=1e-2, seed=1))
    whole.set_state(Q)
    dt = whole.max_dt(0.3)
    parts = Parts(desc, phys, p, 3)
    try:
        parts.set_state(Q)
        assert min(m.max_dt(0.3) for m in parts.meshes) == dt
        for _ in range(3):
            whole.rk_step(0.0, dt)
            for s in range(4):
                parts.stage(fr.FR_RK44, s, dt)
        got = parts.gather([m.get_state() for m in parts.meshes], Q.shape)
        np.testing.assert_array_equal(got, whole.get_state())
    finally:
        parts.close()
        whole.close()


class MixedParts(Parts):
    """Parts of a mesh with prisms: states and residuals are [n_points][5] (hexahedral points,
    then prism points); each part's rows are its elements' point ranges."""

    def __init__(self, desc, phys, p, n_parts, E, Np, Npp):
        super().__init__(desc, phys, p, n_parts)
        self.rows = []
        for h in self.halo:
            eg = np.asarray(h["elem_global"])
            self.rows.append(np.concatenate(
                [e * Np + np.arange(Np) if e < E else E * Np + (e - E) * Npp + np.arange(Npp) for e in eg]))

    def set_state(self, Q):
        for m, rows in zip(self.meshes, self.rows):
            m.set_state(np.ascontiguousarray(Q[rows].reshape(m.shape)))

    def gather(self, arrays, shape):
        out = np.empty(shape)
        for a, rows in zip(arrays, self.rows):
            out[rows] = np.asarray(a).reshape(-1, 5)
        return out


@pytest.mark.parametrize("split", ["checker", "all"])
@pytest.mark.parametrize("precision", [0, 1])
def test_partitioned_mixed_mesh_equals_whole_mesh(split, precision):
    """Hexahedra and prisms across part boundaries (triangular and quadrilateral halo
    interfaces): residual and two RK44 steps equal to the whole mesh's, bit for bit."""
    torch = pytest.importorskip("torch")
    ensure_lib()
    desc = I.hex_box_mesh((4, 4, 3), prisms=split, seed=2)
    phys = I.tgv_physics(Ma=0.2, Re=400.0)
    phys.precision = precision
    p = 3
    with fr.Mesh(desc, phys, p) as whole:
        Q = np.ascontiguousarray(I.tgv_state(whole.solution_points(), Ma=0.2, perturb=1e-2, seed=3))
        whole.set_state(Q)
        R_whole = whole.residual()
        dt = whole.max_dt(0.3)
        parts = MixedParts(desc, phys, p, 3, whole.n_elem, whole.n_pts, whole.n_pts_prism)
        try:
            assert all(h["n_halo"] > 0 for h in parts.halo)
            parts.set_state(Q)
            Rd = [torch.empty(m.shape, dtype=torch.float64, device="cuda") for m in parts.meshes]
            parts.stage(R=Rd)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(parts.gather([r.cpu().numpy() for r in Rd], R_whole.shape), R_whole)
            for _ in range(2):
                whole.rk_step(0.0, dt)
                for st in range(4):
                    parts.stage(fr.FR_RK44, st, dt)
            got = parts.gather([m.get_state() for m in parts.meshes], Q.shape)
            np.testing.assert_array_equal(got, whole.get_state())
        finally:
            parts.close()


def test_part_refusals_and_single_part():
    torch = pytest.importorskip("torch")
    ensure_lib()
    desc = I.hex_box_mesh((3, 3, 2), seed=1)
    phys = I.tgv_physics()
    part = fr.partition(desc, 2, 2)
    with fr.PartMesh(desc, phys, 2, part, 0) as m:
        m.set_state(np.ascontiguousarray(I.tgv_state(m.solution_points())))
        for call in (lambda: m.residual(), lambda: m.rk_stage(0, 0.0, 1e-3),
                     lambda: m.set_closure(np.zeros(9153, np.float32), np.r_[np.zeros(11), np.ones(11), 1.0])):
            with pytest.raises(fr.FRError) as ei:
                call()
            assert ei.value.status == fr.FR_EUNSUPPORTED
        with pytest.raises(fr.FRError) as ei:
            m.phase(1)                         # NULL halo buffers
        assert ei.value.status == fr.FR_EINVAL
    # One part owning everything has no halo and behaves like the whole mesh.
    with fr.PartMesh(desc, phys, 2, np.zeros(18, np.int32), 0) as m, fr.Mesh(desc, phys, 2) as w:
        Q = np.ascontiguousarray(I.tgv_state(w.solution_points()))
        m.set_state(Q)
        w.set_state(Q)
        np.testing.assert_array_equal(m.residual(), w.residual())
