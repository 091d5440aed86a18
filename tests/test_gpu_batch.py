"""Batched persistent RK stages (fr_batch_*) vs the per-mesh path and the oracle (marked gpu)."""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle.hexfr import HexFR

from helpers import assert_state_parity, ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _cases(precision=0):
    """A ragged ensemble: different orders, sizes, orientations, one case with walls."""
    specs = []
    for k, (n, p) in enumerate([(3, 2), (2, 5), (4, 3), (3, 4), (2, 1), (3, 3)]):
        d = I.hex_box_mesh((n, n, n), seed=k, shuffle=True, rotate=True, perturb=0.05 if k % 2 else 0.0)
        specs.append((d, I.tgv_physics(Ma=0.2, Re=300.0), p, k))
    walls = I.hex_box_mesh((3, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, True),
                           wall_tags={1: (I.BC_WALL_ISOTHERMAL, (1.1,)), 2: (I.BC_CHAR_OUTFLOW, (0.7,))}, seed=9, rotate=True)
    specs.append((walls, I.Physics(gamma=1.4, R=1.0, mu=0.02, Pr=0.71, viscous=1), 3, 99))
    for _, ph, _, _ in specs:
        ph.precision = precision
    return specs


def _state(ora, seed, wall):
    if wall:
        X = ora.x
        return np.ascontiguousarray(I.conserved(1 + 0.1 * np.sin(X[..., 0]), 0.2 * np.cos(X[..., 1] * 2 * np.pi),
                                                0.1 + 0 * X[..., 0], 0.05 * np.sin(2 * np.pi * X[..., 2]),
                                                0.7 + 0.02 * X[..., 0], 1.4))
    return np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.2, perturb=1e-2, seed=seed))


def _close(got, want):
    """Same arithmetic in another kernel: equal up to a few ulps (FMA contraction may differ)."""
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-14 * np.abs(want).max())


def _build(specs, stream=0):
    oras, meshes, Qs, dts = [], [], [], []
    for d, ph, p, k in specs:
        ora = HexFR(d, ph, p)
        Q = _state(ora, k, k == 99)
        m = fr.Mesh(d, ph, p, stream=stream)
        m.set_state(Q)
        oras.append(ora)
        meshes.append(m)
        Qs.append(Q)
        dts.append(0.5 * ora.max_dt(Q, 0.3))
    return oras, meshes, Qs, dts


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_step_equals_per_mesh_steps(precision):
    specs = _cases(precision)
    _, single, Qs, dts = _build(specs)
    _, batched, _, _ = _build(specs)
    for m, dt in zip(single, dts):
        for _ in range(2):
            m.rk_step(0.0, dt)
    with fr.Batch(batched) as b:
        b.set_dt(dts)
        for _ in range(2):
            b.rk_step(0.0)
    for a, c in zip(single, batched):
        _close(c.get_state(), a.get_state())


def test_batch_per_case_executor_equals_per_mesh():
    specs = _cases(1)
    _, single, Qs, dts = _build(specs)
    _, batched, _, _ = _build(specs)
    for m, dt in zip(single, dts):
        m.rk_step(0.0, dt)
    with fr.Batch(batched) as b:
        b.select(1)
        b.set_dt(dts)
        b.rk_step(0.0)
    for a, c in zip(single, batched):
        np.testing.assert_array_equal(c.get_state(), a.get_state())


def test_batch_matches_oracle():
    specs = _cases(0)[:3]
    oras, meshes, Qs, dts = _build(specs)
    with fr.Batch(meshes) as b:
        b.set_dt(dts)
        b.rk_step(0.0)
    for ora, m, Q, dt in zip(oras, meshes, Qs, dts):
        assert_state_parity(m.get_state(), ora.rk44_step(Q, 0.0, dt), ora.residual(Q, magnitude=True), dt)


def test_batch_graphs_on_stream_and_tuning():
    torch = pytest.importorskip("torch")
    specs = _cases(1)
    s = torch.cuda.Stream()
    _, ref, Qs, dts = _build(specs)
    _, meshes, _, _ = _build(specs, stream=s.cuda_stream)
    with fr.Batch(ref) as b0:
        b0.set_dt(dts)
        for _ in range(3):
            b0.rk_step(0.0)
    with fr.Batch(meshes) as b:
        b.tune()                     # times configurations, then restores every case to U_n
        info = b.info()
        assert info["block"] in (256, 512) and info["grid"] >= info["blocks_per_sm"]
        b.set_dt(dts)
        for _ in range(3):           # stage graphs captured on the first step, replayed after
            b.rk_step(0.0)
        s.synchronize()
    for a, c in zip(ref, meshes):
        _close(c.get_state(), a.get_state())


def test_batch_barrier_timeout_reports_error():
    """One block leaves before the first grid barrier; the others give up after a short bounded
    wait and the call reports FR_ETIMEOUT (the context stays usable)."""
    torch = pytest.importorskip("torch")
    specs = _cases(0)[:2]
    _, meshes, _, dts = _build(specs)
    b = fr.Batch(meshes)
    b.set_dt(dts)
    b.debug(0, 20000)
    with pytest.raises(fr.FRError) as ei:
        b.rk_stage(0)
    assert ei.value.status == fr.FR_ETIMEOUT
    with pytest.raises(fr.FRError) as ei2:
        meshes[0].residual()
    assert ei2.value.status == fr.FR_ETIMEOUT
    b.close()
    x = torch.ones(4, device="cuda")
    assert float((x * 2).sum().item()) == 8.0     # the device still works


def _mixed_type_specs():
    """Hexahedral, prismatic and curved mixed meshes of orders 2..7 (p = 7 prisms need 512-thread
    blocks)."""
    return [(I.hex_box_mesh((3, 3, 2), prisms="checker", seed=1, rotate=True, shuffle=True, perturb=0.05), 3),
            (I.hex_box_mesh((2, 2, 2), prisms="all", seed=2, rotate=True), 5),
            (I.curved_box_mesh((2, 2, 2), prisms="checker", warp=0.1, seed=3, rotate=True), 4),
            (I.hex_box_mesh((3, 3, 3), seed=4, rotate=True), 2),
            (I.curved_box_mesh((2, 2, 2), prisms="all", warp=0.1, seed=5), 7)]


def _mixed_type_build(precision):
    from oracle.mixedfr import MixedFR
    oras, meshes, Qs = [], [], []
    for k, (d, p) in enumerate(_mixed_type_specs()):
        ph = I.tgv_physics(Ma=0.2, Re=300.0)
        ph.precision = precision
        ora = MixedFR(d, I.tgv_physics(Ma=0.2, Re=300.0), p)
        Q = [np.ascontiguousarray(I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=k)) for x in ora.x]
        m = fr.Mesh(d, ph, p)
        m.set_state(np.ascontiguousarray(np.concatenate([q.reshape(-1, 5) for q in Q])))
        oras.append(ora)
        meshes.append(m)
        Qs.append(Q)
    return oras, meshes, Qs


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_batch_mixed_element_types(precision, mode):
    dt = 1e-3
    _, single, _ = _mixed_type_build(precision)
    oras, batched, Qs = _mixed_type_build(precision)
    for m in single:
        for _ in range(2):
            m.rk_step(0.0, dt)
    with fr.Batch(batched) as b:
        b.select(mode)
        b.set_dt([dt] * len(batched))
        assert b.info()["block"] == 512
        for _ in range(2):
            b.rk_step(0.0)
    for a, c in zip(single, batched):
        if mode == 1:
            np.testing.assert_array_equal(c.get_state(), a.get_state())
        else:
            _close(c.get_state(), a.get_state())
    if precision == 0 and mode == 0:
        # one case against the oracle's RK44 (two steps)
        ora, m, Q = oras[0], batched[0], Qs[0]
        S = np.concatenate([s.reshape(-1, 5) for s in ora.residual(Q, magnitude=True)])
        for _ in range(2):
            k1 = ora.residual(Q)
            k2 = ora.residual([q + 0.5 * dt * k for q, k in zip(Q, k1)])
            k3 = ora.residual([q + 0.5 * dt * k for q, k in zip(Q, k2)])
            k4 = ora.residual([q + dt * k for q, k in zip(Q, k3)])
            Q = [q + dt / 6.0 * (a + 2 * b_ + 2 * c + e) for q, a, b_, c, e in zip(Q, k1, k2, k3, k4)]
        assert_state_parity(m.get_state(), np.concatenate([q.reshape(-1, 5) for q in Q]), S, 2 * dt)


def test_batch_mixed_types_tuning_restores_state():
    oras, meshes, Qs = _mixed_type_build(1)
    before = [m.get_state().copy() for m in meshes]
    with fr.Batch(meshes) as b:
        b.set_dt([1e-3] * len(meshes))
        b.tune()
        info = b.info()
        assert info["mode"] in (0, 1) and info["n_points"] == sum(m.n_points for m in meshes)
        for m, q in zip(meshes, before):
            np.testing.assert_array_equal(m.get_state(), q)
        b.rk_step(0.0)
    for m in meshes:
        assert np.isfinite(m.get_state()).all()
