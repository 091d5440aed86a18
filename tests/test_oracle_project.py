"""Pins of the oracle's order projection (CPU): exact on polynomials of degree <= min(p, q), the
projection error is orthogonal to the target space, projecting down then up reproduces the
truncation, and up then down is the identity."""
import numpy as np
import pytest

from oracle import project as PJ
from oracle.basis import Basis1D
from oracle.mixedfr import MixedFR
from oracle.tri import Tri
from paper_2308_06605_gb300 import inputs as I


@pytest.mark.parametrize("p,q", [(1, 3), (3, 1), (2, 5), (4, 2), (3, 3), (7, 4)])
def test_polynomial_exactness(p, q):
    # Affine elements (a box, the local vertex order may rotate): a physical polynomial of degree
    # k = min(p, q) is a reference polynomial of the same degree in every element.
    d = I.hex_box_mesh((2, 2, 1), prisms="checker", seed=1, rotate=True)
    ph = I.tgv_physics()
    mp, mq = MixedFR(d, ph, p), MixedFR(d, ph, q)
    k = min(p, q)
    f = lambda x: (x[..., 0] ** k + 0.3 * x[..., 1] ** max(k - 1, 0) * x[..., 2] + 0.7)[..., None] * np.ones(5)  # noqa: E731
    for got, want in zip(PJ.project([f(x) for x in mp.x], p, q), [f(x) for x in mq.x]):
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("p,q", [(4, 2), (5, 3)])
def test_error_orthogonal_to_target_space(p, q):
    # hexahedron, one element, reference coordinates: integrate (f - Pf) * phi with the order-p rule
    b = Basis1D(p)
    x = b.nodes
    f = np.exp(x) * np.cos(2 * x)
    g = PJ.line_transfer(p, q) @ f                      # values of Pf at the order-q points
    back = PJ.line_transfer(q, p) @ g                   # Pf (degree q) at the order-p points, exact
    for k in range(q + 1):
        phi = np.polynomial.legendre.legval(x, np.eye(q + 1)[k])
        assert abs(np.sum(b.weights * (f - back) * phi)) < 1e-14
    # triangle: the same with the order-p triangle's exact mass matrix
    Tp = Tri(p)
    rs = Tp.rs
    F = np.exp(rs[:, 0]) * np.sin(rs[:, 1] + 0.3)
    back = PJ.tri_transfer(q, p) @ (PJ.tri_transfer(p, q) @ F)
    Pq = Tri(q)
    for n in range(Pq.Nt):
        phi = Pq.interp(rs)[:, n]
        assert abs(phi @ Tp.M @ (F - back)) < 1e-13


def test_up_then_down_is_identity():
    for p, q in ((2, 4), (3, 6)):
        np.testing.assert_allclose(PJ.line_transfer(q, p) @ PJ.line_transfer(p, q), np.eye(p + 1), atol=1e-13)
        Tt = PJ.tri_transfer(q, p) @ PJ.tri_transfer(p, q)
        np.testing.assert_allclose(Tt, np.eye(Tt.shape[0]), atol=1e-12)
