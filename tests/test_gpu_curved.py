"""Quadratic (curved) elements on the GPU vs the mixed-element oracle (marked gpu).

27-node hexahedra and 18-node prisms with conservative-curl metrics, warped periodic boxes
(rotated, shuffled), orders 1..7: residual per entry <= 1e-12 S (FP64), <= 1e-9 S (mixed);
free stream on the GPU within the oracle's rounding bar 1e-13 (p+1)^2 max|F| / h_min; walls
through curved faces; RK steps.
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


def _phys(precision=0):
    ph = I.tgv_physics(Ma=0.2, Re=300.0)
    ph.precision = precision
    return ph


@pytest.mark.parametrize("p,prisms", [(1, "checker"), (2, None), (3, "all"), (4, "checker"), (5, None),
                                      (6, "checker"), (7, "all")])
def test_curved_residual(p, prisms):
    d = I.curved_box_mesh((2, 2, 2), prisms=prisms, warp=0.15, seed=p, rotate=True, shuffle=True)
    ora = MixedFR(d, _phys(), p)
    Qs = [np.ascontiguousarray(I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=p)) for x in ora.x]
    Ro, So = flat(ora.residual(Qs)), flat(ora.residual(Qs, magnitude=True))
    for prec, rel in ((0, 1e-12), (1, 1e-9)):
        with fr.Mesh(d, _phys(prec), p) as g:
            np.testing.assert_allclose(g.solution_points().reshape(-1, 3), flat(ora.x), rtol=0, atol=1e-12 * 2 * np.pi)
            g.set_state(flat(Qs))
            R = g.residual()
        assert_residual_parity(R.reshape(-1, 5), Ro, So, rel=rel)


@pytest.mark.parametrize("p", [2, 4, 7])
def test_curved_free_stream(p):
    d = I.curved_box_mesh((3, 2, 2), prisms="checker", warp=0.15, seed=p, rotate=True, shuffle=True)
    ph = I.Physics(gamma=1.4, R=1.0, mu=0.0, viscous=0)
    ora = MixedFR(d, ph, p)
    scale = (0.3 ** 2 + 1 / 1.4) / min(h.min() for h in ora.h if len(h))
    with fr.Mesh(d, ph, p) as g:
        g.set_state(np.ascontiguousarray(I.uniform_state((g.n_points,))))
        R = g.residual()
    assert np.abs(R).max() <= 1e-13 * (p + 1) ** 2 * scale


def test_curved_walls_and_rk_steps():
    p = 3
    d = I.curved_box_mesh((2, 2, 3), hi=(1.0, 1.0, 1.5), periodic=(True, True, False), prisms="checker", warp=0.1,
                          seed=2, rotate=True, shuffle=True,
                          wall_tags={5: (I.BC_DIRICHLET, tuple(I.conserved(1.0, 0.1, 0.1, 0.0, 1.0, 1.4))),
                                     6: (I.BC_DIRICHLET, tuple(I.conserved(1.05, 0.0, 0.1, 0.05, 1.03, 1.4)))})
    ph = I.Physics(gamma=1.4, R=1.0, mu=0.02, Pr=0.71, viscous=1)
    ora = MixedFR(d, ph, p)

    def st(X):
        return I.conserved(1 + 0.1 * np.sin(2 * np.pi * X[..., 0]), 0.2 * np.cos(2 * np.pi * X[..., 1]),
                           0.1 + 0 * X[..., 0], 0.05 * np.sin(X[..., 2]), 1.0 + 0.02 * X[..., 2], 1.4)
    Qs = [np.ascontiguousarray(st(x)) for x in ora.x]
    So = flat(ora.residual(Qs, magnitude=True))
    with fr.Mesh(d, ph, p) as g:
        g.set_state(flat(Qs))
        assert_residual_parity(g.residual(), flat(ora.residual(Qs)), So, rel=1e-12)
        dt = 0.25 * g.max_dt(0.3)
        for s in range(2):
            g.rk_step(s * dt, dt)
        Qg = g.get_state()
    Q = Qs
    for _ in range(2):
        k1 = ora.residual(Q)
        k2 = ora.residual([q + 0.5 * dt * k for q, k in zip(Q, k1)])
        k3 = ora.residual([q + 0.5 * dt * k for q, k in zip(Q, k2)])
        k4 = ora.residual([q + dt * k for q, k in zip(Q, k3)])
        Q = [q + dt / 6.0 * (a + 2 * b + 2 * c + e) for q, a, b, c, e in zip(Q, k1, k2, k3, k4)]
    assert_state_parity(Qg, flat(Q), So, 2 * dt, rel=1e-12)
