"""GPU FP64 path vs the oracle, through the C ABI (marked gpu).

Residual bar, per entry: |R_gpu - R_oracle| <= 1e-12 * S, where S is the oracle's magnitude
scale of that entry (the sum of the magnitudes of the terms of Eq. 3 that form it).  States after
RK steps: |Q_gpu - Q_oracle| <= 1e-12 * (|Q| + T S), T the elapsed time.
"""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle.basis import Basis1D
from oracle.hexfr import HexFR, trilinear_geometry

from helpers import assert_residual_parity, assert_state_parity, ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _pair(desc, phys, p, state):
    ora = HexFR(desc, phys, p)
    Q = state(ora.x)
    gpu = fr.Mesh(desc, phys, p)
    return ora, gpu, np.ascontiguousarray(Q)


def test_solution_points_match_oracle():
    d = I.hex_box_mesh((3, 3, 3), seed=3, shuffle=True, rotate=True, perturb=0.1)
    ora = HexFR(d, I.tgv_physics(), 3)
    with fr.Mesh(d, I.tgv_physics(), 3) as g:
        np.testing.assert_allclose(g.solution_points(), ora.x, rtol=0, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_residual_parity_all_orders(p):
    """Shuffled, randomly rotated, perturbed-trilinear periodic mesh; perturbed TGV; NS + BR2."""
    n = 4 if p <= 4 else 3
    d = I.hex_box_mesh((n, n, n), seed=p, shuffle=True, rotate=True, perturb=0.1)
    phys = I.tgv_physics(Ma=0.2, Re=200.0)
    ora, g, Q = _pair(d, phys, p, lambda x: I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=p))
    g.set_state(Q)
    assert_residual_parity(g.residual(), ora.residual(Q), ora.residual(Q, magnitude=True))
    g.close()


def test_residual_parity_config_8cube_p3_tgv():
    """The 8^3, p = 3 TGV at Ma 0.1, Re 1600, stored unstructured (shuffled + rotated)."""
    d = I.hex_box_mesh((8, 8, 8), seed=0, shuffle=True, rotate=True)
    phys = I.tgv_physics()
    for seed in range(3):
        ora, g, Q = _pair(d, phys, 3, lambda x: I.tgv_state(x, Ma=0.1, perturb=1e-3, seed=seed))
        g.set_state(Q)
        assert_residual_parity(g.residual(), ora.residual(Q), ora.residual(Q, magnitude=True))
        g.close()


def test_euler_parity_and_free_stream():
    d = I.hex_box_mesh((3, 4, 2), seed=5, rotate=True, perturb=0.15)
    phys = I.Physics(gamma=1.4, R=1.0, mu=0.0, viscous=0)
    ora, g, Q = _pair(d, phys, 4, lambda x: I.isentropic_vortex_state(x, centre=(3.0, 3.0), period=(2 * np.pi,) * 2))
    g.set_state(Q)
    assert_residual_parity(g.residual(), ora.residual(Q), ora.residual(Q, magnitude=True))
    U = I.uniform_state(ora.x.shape[:2])
    g.set_state(np.ascontiguousarray(U))
    R = g.residual()
    Fmax = 1.5     # |F| of the uniform state is below this
    assert np.abs(R).max() <= 1e-13 * Fmax / ora.h.min()
    g.close()


def test_conservation_on_gpu():
    d = I.hex_box_mesh((4, 4, 4), seed=9, shuffle=True, rotate=True, perturb=0.1)
    phys = I.tgv_physics(Ma=0.3, Re=300.0)
    ora, g, Q = _pair(d, phys, 3, lambda x: I.tgv_state(x, Ma=0.3, perturb=1e-2, seed=2))
    g.set_state(Q)
    R = g.residual()
    s = np.abs(ora.integrate(R))
    a = np.einsum('m,em,emv->v', ora.W, ora.detJ, np.abs(R))
    assert np.all(s <= 1e-12 * a)
    g.close()


def test_rk44_ten_steps_config_8cube_p3():
    """10 RK44 steps at CFL 0.3 on the 8^3 p = 3 TGV: GPU state vs oracle state."""
    d = I.hex_box_mesh((8, 8, 8), seed=0, shuffle=True, rotate=True)
    phys = I.tgv_physics()
    ora, g, Q = _pair(d, phys, 3, lambda x: I.tgv_state(x, Ma=0.1))
    g.set_state(Q)
    dt_g = g.max_dt(0.3)
    dt_o = ora.max_dt(Q, 0.3)
    assert abs(dt_g - dt_o) <= 1e-14 * dt_o
    Qo = Q.copy()
    t = 0.0
    for _ in range(10):
        g.rk_step(t, dt_o)
        Qo = ora.rk44_step(Qo, t, dt_o)
        t += dt_o
    Qg = g.get_state()
    assert_state_parity(Qg, Qo, ora.residual(Q, magnitude=True), t)
    g.close()


@pytest.mark.parametrize("kinds", [
    ((I.BC_WALL_ISOTHERMAL, (1.1,)), (I.BC_CHAR_OUTFLOW, (0.7,))),
    ((I.BC_CHAR_INFLOW, (0.9, 1.05, 1.0, 0.2, 0.0)), (I.BC_WALL_ISOTHERMAL, (0.9,))),
    ((I.BC_DIRICHLET, (1.0, 0.1, 0.0, 0.0, 1.8)), (I.BC_CHAR_OUTFLOW, (0.68,)))])
@pytest.mark.parametrize("p", [2, 4])
def test_boundary_conditions_parity(kinds, p):
    """Walls, characteristic inflow/outflow and Dirichlet faces on a rotated, perturbed mesh."""
    d = I.hex_box_mesh((3, 2, 2), hi=(2.0, 1.0, 1.0), periodic=(False, True, True),
                       wall_tags={1: kinds[0], 2: kinds[1]}, seed=3, rotate=True, shuffle=True, perturb=0.1)
    phys = I.Physics(gamma=1.4, R=1.0, mu=0.02, Pr=0.71, viscous=1)

    def st(X):
        return I.conserved(1 + 0.1 * np.sin(X[..., 0]), 0.2 * np.cos(X[..., 1] * 2 * np.pi),
                           0.1 + 0 * X[..., 0], 0.05 * np.sin(2 * np.pi * X[..., 2]), 0.7 + 0.02 * X[..., 0], 1.4)
    ora, g, Q = _pair(d, phys, p, st)
    g.set_state(Q)
    assert_residual_parity(g.residual(), ora.residual(Q), ora.residual(Q, magnitude=True))
    g.close()


def test_device_pointers_and_state_roundtrip():
    torch = pytest.importorskip("torch")
    d = I.hex_box_mesh((3, 3, 3), seed=1, rotate=True)
    phys = I.tgv_physics(Ma=0.2, Re=200.0)
    ora, g, Q = _pair(d, phys, 2, lambda x: I.tgv_state(x, Ma=0.2, perturb=1e-2))
    Qd = torch.from_numpy(Q).cuda()
    g.set_state(Qd)
    Rd = torch.empty_like(Qd)
    g.residual(out=Rd)
    torch.cuda.synchronize()
    Rh = g.residual()
    np.testing.assert_array_equal(Rd.cpu().numpy(), Rh)
    back = torch.empty_like(Qd)
    g.get_state(out=back)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(back.cpu().numpy(), Q)
    g.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_resume_is_bit_identical(precision):
    """Checkpoint at a step boundary: get_state after one RK44 step, a new mesh set_state from it
    and two more steps give exactly the state of three uninterrupted steps (the FP64 state is the
    whole RK state at a step boundary; the double-float copies are rebuilt from it the same way)."""
    d = I.hex_box_mesh((3, 3, 2), seed=5, rotate=True, shuffle=True, perturb=0.1)
    phys = I.tgv_physics(Ma=0.2, Re=300.0)
    phys.precision = precision
    ora = HexFR(d, I.tgv_physics(Ma=0.2, Re=300.0), 3)
    Q0 = np.ascontiguousarray(I.tgv_state(ora.x, Ma=0.2, perturb=1e-2, seed=5))
    dt = 0.5 * ora.max_dt(Q0, 0.3)
    with fr.Mesh(d, phys, 3) as a:
        a.set_state(Q0)
        for s in range(3):
            a.rk_step(s * dt, dt)
        Qa = a.get_state()
    with fr.Mesh(d, phys, 3) as b:
        b.set_state(Q0)
        b.rk_step(0.0, dt)
        Q1 = b.get_state()
    with fr.Mesh(d, phys, 3) as c:
        c.set_state(Q1)
        for s in range(1, 3):
            c.rk_step(s * dt, dt)
        Qc = c.get_state()
    assert np.array_equal(Qa, Qc)


def test_nonfinite_state_reported():
    d = I.hex_box_mesh((2, 2, 2))
    phys = I.tgv_physics()
    ora, g, Q = _pair(d, phys, 2, lambda x: I.tgv_state(x))
    Q[1, 3, 4] = np.nan
    g.set_state(Q)
    for s in range(3):
        g.rk_stage(s, 0.0, 1e-3)
    with pytest.raises(fr.FRError) as ei:
        g.rk_stage(3, 0.0, 1e-3)
    assert ei.value.status == fr.FR_ENONFINITE
    g.close()


@pytest.mark.parametrize("precision,rel", [(0, 1e-12), (1, 1e-9)])
def test_full_size_64cube_p4_sampled(precision, rel):
    """The 64^3, p = 4 TGV (32.8 M points) in the benchmark's launch configuration, both
    precisions (the double-float one is the headline path), checked on sampled elements: BR2 is
    compact, so an element's residual depends only on itself and its six face neighbours; the
    oracle evaluates each sample on a 3x3x3 periodic patch holding the same data and geometry,
    whose centre element is the sample."""
    n, p = 64, 4
    L = 2 * np.pi
    h = L / n
    d = I.hex_box_mesh((n, n, n))
    phys = I.tgv_physics()
    gphys = I.tgv_physics()
    gphys.precision = precision
    g = fr.Mesh(d, gphys, p)
    # Solution points from the oracle's own geometry (never from the library).
    xi = Basis1D(p).nodes
    K, Jj, Ii = np.meshgrid(xi, xi, xi, indexing="ij")
    ref = np.stack([Ii.ravel(), Jj.ravel(), K.ravel()], axis=1)
    x, _, _ = trilinear_geometry(d.xyz[d.hex], ref)
    Q = np.ascontiguousarray(I.tgv_state(x, Ma=0.1, perturb=1e-3, seed=4))
    del x
    g.set_state(Q)
    R = g.residual()
    rng = np.random.default_rng(0)
    idx = [(0, 0, 0), (n - 1, n - 1, n - 1), (n - 1, 0, 5)] + [tuple(rng.integers(0, n, 3)) for _ in range(9)]
    Np = (p + 1) ** 3
    for (i, j, k) in idx:
        patch = I.hex_box_mesh((3, 3, 3), lo=((i - 1) * h, (j - 1) * h, (k - 1) * h),
                               hi=((i + 2) * h, (j + 2) * h, (k + 2) * h))
        ora = HexFR(patch, phys, p)
        Qp = np.empty((27, Np, 5))
        for kk in range(3):
            for jj in range(3):
                for ii in range(3):
                    e_full = ((i - 1 + ii) % n) + n * (((j - 1 + jj) % n) + n * ((k - 1 + kk) % n))
                    Qp[ii + 3 * (jj + 3 * kk)] = Q[e_full]
        Rp = ora.residual(Qp)
        Sp = ora.residual(Qp, magnitude=True)
        e_c = i + n * (j + n * k)
        assert_residual_parity(R[e_c], Rp[13], Sp[13], rel=rel)
    # Discrete conservation at full size: quadrature weights (library Gauss-Legendre rule) on
    # congruent affine cubes, so the constant |J| drops out.
    w = np.polynomial.legendre.leggauss(p + 1)[1]
    W = np.kron(w, np.kron(w, w))
    s = np.abs(np.einsum('m,emv->v', W, R))
    a = np.einsum('m,emv->v', W, np.abs(R))
    # Double-float: the per-entry bar is 1e-9 of the magnitude scale S, and at Ma 0.1 S exceeds |R|
    # by up to ~1e2 (cancelling terms), so the sum is held to 1e-7 of sum |W R|.
    assert np.all(s <= (1e-12 if precision == 0 else 1e-7) * a), s / a
    g.close()
