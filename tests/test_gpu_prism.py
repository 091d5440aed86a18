"""Prisms: mixed hexahedral/prismatic meshes on the GPU vs the mixed-element FP64 oracle (marked gpu).

Bars as for hexahedra: per entry |R_gpu - R_oracle| <= 1e-12 S on the FP64 path and <= 1e-9 S
(normwise <= 1e-6) on the double-float path, S = the oracle's magnitude scale of the entry's sum
(Eq. 3); states after RK44 steps within 1e-12 (|Q| + t S).  Meshes: periodic boxes whose columns
are all, or every other one, split into two prisms, with rotated local vertex orders (all six
prism and 24 hexahedron orientations appear), shuffled element order and perturbed interior
nodes; Dirichlet boundaries through triangular faces; orders 1..7.
"""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle.mixedfr import MixedFR

from helpers import assert_residual_parity, assert_state_parity, ensure_lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def flat(arrs):
    return np.concatenate([np.asarray(a).reshape(-1, np.asarray(a).shape[-1]) for a in arrs])


def _phys(precision=0, viscous=True):
    ph = I.tgv_physics(Ma=0.2, Re=300.0)
    ph.precision = precision
    if not viscous:
        ph.viscous, ph.mu = 0, 0.0
    return ph


def _mesh(n, prisms, seed, perturb=0.1, **kw):
    return I.hex_box_mesh(n, prisms=prisms, seed=seed, rotate=True, shuffle=True, perturb=perturb, **kw)


def _state(ora, seed):
    return [np.ascontiguousarray(I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=seed)) for x in ora.x]


CASES = [(1, (3, 3, 2), "all"), (2, (3, 3, 2), "checker"), (3, (3, 2, 2), "all"), (4, (3, 3, 2), "checker"),
         (5, (2, 2, 2), "all"), (6, (2, 2, 2), "checker"), (7, (2, 2, 2), "checker")]


@pytest.mark.parametrize("p,n,prisms", CASES)
def test_points_and_fp64_residual(p, n, prisms):
    d = _mesh(n, prisms, seed=p)
    ph = _phys()
    ora = MixedFR(d, ph, p)
    Qs = _state(ora, p)
    with fr.Mesh(d, ph, p) as g:
        assert g.n_prism == len(d.prism) and g.n_elem == len(d.hex)
        x = g.solution_points()
        # Same point set and order as the oracle's definition (hexahedra, then prisms).
        np.testing.assert_allclose(x, flat(ora.x), rtol=0, atol=1e-12 * 2 * np.pi)
        g.set_state(flat(Qs))
        R = g.residual()
    assert_residual_parity(R, flat(ora.residual(Qs)), flat(ora.residual(Qs, magnitude=True)), rel=1e-12)


@pytest.mark.parametrize("p", [2, 4])
def test_euler_residual(p):
    d = _mesh((3, 3, 2), "checker", seed=10 + p)
    ph = _phys(viscous=False)
    ora = MixedFR(d, ph, p)
    Qs = _state(ora, p)
    with fr.Mesh(d, ph, p) as g:
        g.set_state(flat(Qs))
        R = g.residual()
    assert_residual_parity(R, flat(ora.residual(Qs)), flat(ora.residual(Qs, magnitude=True)), rel=1e-12)


@pytest.mark.parametrize("prisms", ["all", "checker"])
def test_dirichlet_through_triangular_faces(prisms):
    hi = (1.0, 1.0, 1.5)
    ext = (1.0, 0.1, -0.05, 0.02, 2.6)

    def st(X):
        return I.conserved(1 + 0.1 * np.sin(2 * np.pi * X[..., 0]), 0.2 * np.cos(2 * np.pi * X[..., 1]),
                           0.1 + 0 * X[..., 0], 0.05 * np.sin(X[..., 2]), 1.0 + 0.02 * X[..., 2], 1.4)
    d = I.hex_box_mesh((2, 2, 3), hi=hi, periodic=(True, True, False), prisms=prisms, seed=4, rotate=True,
                       shuffle=True, perturb=0.1,
                       wall_tags={5: (I.BC_DIRICHLET, ext), 6: (I.BC_DIRICHLET, (0.9, 0.0, 0.1, -0.1, 2.2))})
    ph = I.Physics(gamma=1.4, R=1.0, mu=0.02, Pr=0.71, viscous=1)
    ora = MixedFR(d, ph, 3)
    Qs = [np.ascontiguousarray(st(x)) for x in ora.x]
    for prec, rel in ((0, 1e-12), (1, 1e-9)):
        ph.precision = prec
        with fr.Mesh(d, ph, 3) as g:
            g.set_state(flat(Qs))
            R = g.residual()
        assert_residual_parity(R, flat(ora.residual(Qs)), flat(ora.residual(Qs, magnitude=True)), rel=rel)


@pytest.mark.parametrize("p", [1, 3, 4, 6])
def test_mixed_precision_residual(p):
    d = _mesh((3, 3, 2) if p <= 4 else (2, 2, 2), "checker", seed=20 + p)
    ph = _phys(precision=1)
    ora = MixedFR(d, _phys(), p)
    Qs = _state(ora, p)
    with fr.Mesh(d, ph, p) as g:
        g.set_state(flat(Qs))
        R = g.residual()
    Ro = flat(ora.residual(Qs))
    assert_residual_parity(R, Ro, flat(ora.residual(Qs, magnitude=True)), rel=1e-9)
    norm = np.abs(R - Ro).max(axis=0) / np.abs(Ro).max(axis=0)
    assert np.all(norm <= 1e-6), norm


def _rk44(ora, Qs, dt, n):
    for _ in range(n):
        k1 = ora.residual(Qs)
        k2 = ora.residual([q + 0.5 * dt * k for q, k in zip(Qs, k1)])
        k3 = ora.residual([q + 0.5 * dt * k for q, k in zip(Qs, k2)])
        k4 = ora.residual([q + dt * k for q, k in zip(Qs, k3)])
        Qs = [q + dt / 6.0 * (a + 2 * b + 2 * c + e) for q, a, b, c, e in zip(Qs, k1, k2, k3, k4)]
    return Qs


@pytest.mark.parametrize("precision,rel", [(0, 1e-12), (1, 1e-9)])
def test_rk44_steps(precision, rel):
    d = _mesh((3, 3, 2), "checker", seed=7)
    p = 3
    ora = MixedFR(d, _phys(), p)
    Qs = _state(ora, 3)
    with fr.Mesh(d, _phys(precision), p) as g:
        g.set_state(flat(Qs))
        dt = 0.5 * g.max_dt(0.3)
        for s in range(3):
            g.rk_step(s * dt, dt)
        Qg = g.get_state()
    assert_state_parity(Qg, flat(_rk44(ora, Qs, dt, 3)), flat(ora.residual(Qs, magnitude=True)), 3 * dt, rel=rel)


def test_max_dt_formula():
    """dt = cfl min_e h_e / ((2p+1) max(|u| + c)), h_e = volume^(1/3) by the elements' quadrature."""
    d = _mesh((3, 3, 2), "checker", seed=8)
    p = 3
    ph = _phys()
    ora = MixedFR(d, ph, p)
    Qs = _state(ora, 8)
    lam = []
    for Q in Qs:
        rho = Q[..., 0]
        u = Q[..., 1:4] / rho[..., None]
        pr = (ph.gamma - 1) * (Q[..., 4] - 0.5 * rho * (u * u).sum(-1))
        lam.append((np.linalg.norm(u, axis=-1) + np.sqrt(ph.gamma * pr / rho)).max(axis=1))
    want = 0.4 * min((h / ((2 * p + 1) * l)).min() for h, l in zip(ora.h, lam))
    with fr.Mesh(d, ph, p) as g:
        g.set_state(flat(Qs))
        assert abs(g.max_dt(0.4) - want) <= 1e-12 * want


def test_free_stream_on_perturbed_mixed_mesh():
    d = _mesh((3, 3, 2), "checker", seed=9, perturb=0.15)
    ph = _phys(viscous=False)
    with fr.Mesh(d, ph, 4) as g:
        x = g.solution_points()
        g.set_state(np.ascontiguousarray(I.uniform_state(x.shape[:1])))
        R = g.residual()
    # Straight-sided elements: the discrete metric identities hold, so uniform flow is steady.
    assert np.abs(R).max() <= 1e-10


def test_prism_meshes_reject_closure_and_static():
    torch = pytest.importorskip("torch")
    d = _mesh((2, 2, 2), "checker", seed=11)
    ph = _phys()
    with fr.Mesh(d, ph, 2) as g:
        with pytest.raises(fr.FRError, match="FR_EUNSUPPORTED"):
            g.set_closure(np.zeros(9153, np.float32), np.concatenate([np.zeros(11), np.ones(12)]).astype(np.float32))
        Q = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        with pytest.raises(fr.FRError, match="FR_EUNSUPPORTED"):
            g.residual_static(Q, torch.empty_like(Q))
