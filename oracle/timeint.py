"""Explicit Runge-Kutta integrators on a residual function (oracle; test infrastructure only).

The paper advances the semi-discretisation with an explicit strong-stability-preserving RK method
(citing Ketcheson 2008).  Written out here, on lists of arrays (one per element type):
  rk44      classical four-stage fourth-order RK;
  ssprk33   the three-stage third-order SSP scheme in Shu-Osher form (SSP coefficient 1);
  ssprk104  Ketcheson's ten-stage fourth-order SSP scheme in its two-register form (SSP
            coefficient 6): five forward-Euler substeps of dt/6, a recombination of the two
            registers, four more substeps and a final combination.
"""
from __future__ import annotations


def _axpy(a, X, b, Y):
    return [a * x + b * y for x, y in zip(X, Y)]


def rk44(f, Q, dt):
    k1 = f(Q)
    k2 = f(_axpy(1.0, Q, 0.5 * dt, k1))
    k3 = f(_axpy(1.0, Q, 0.5 * dt, k2))
    k4 = f(_axpy(1.0, Q, dt, k3))
    return [q + dt / 6.0 * (a + 2 * b + 2 * c + d) for q, a, b, c, d in zip(Q, k1, k2, k3, k4)]


def ssprk33(f, Q, dt):
    u1 = _axpy(1.0, Q, dt, f(Q))
    u2 = _axpy(0.75, Q, 0.25, _axpy(1.0, u1, dt, f(u1)))
    return _axpy(1.0 / 3.0, Q, 2.0 / 3.0, _axpy(1.0, u2, dt, f(u2)))


def ssprk104(f, Q, dt):
    q1, q2 = list(Q), list(Q)
    for _ in range(5):
        q1 = _axpy(1.0, q1, dt / 6.0, f(q1))
    q2 = _axpy(1.0 / 25.0, q2, 9.0 / 25.0, q1)
    q1 = _axpy(15.0, q2, -5.0, q1)
    for _ in range(4):
        q1 = _axpy(1.0, q1, dt / 6.0, f(q1))
    k = f(q1)
    return [b + 0.6 * a + 0.1 * dt * c for a, b, c in zip(q1, q2, k)]


SCHEMES = {"rk44": rk44, "ssprk33": ssprk33, "ssprk104": ssprk104}
STAGES = {"rk44": 4, "ssprk33": 3, "ssprk104": 10}
