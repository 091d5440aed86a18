"""Pins of the oracle's quadratic (curved) elements with conservative-curl metrics (CPU).

- Shape functions: nodal, partition of unity, exact on quadratics.
- Straight-sided elements written with 27/18 nodes: for p >= 2 the curl metrics equal the
  analytic adjugate exactly (the interpolated quantities have degree <= 2), so the residual
  equals the one of the same mesh given with 8/6 nodes.
- Curved meshes: the discrete metric identities sum_d D_d S[d][n] = 0, agreement of the two
  sides' normals, free-stream preservation, discrete conservation, orientation / shuffle
  invariance; on a general quadratic element the curl metrics equal the analytic adjugate for
  p >= 4 (exact interpolation of the degree-4 products) and not below.
Rounding tolerances scale like the derivative matrices, (p + 1)^2.
"""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import curved as C
from oracle.mixedfr import MixedFR
from paper_2308_06605_gb300 import inputs as I

PH = I.tgv_physics(Ma=0.2, Re=300.0)


@pytest.mark.parametrize("kind", ["hex", "prism"])
def test_shape_functions(kind):
    shape, ref = (C.hex27_shape, C.HEX27) if kind == "hex" else (C.prism18_shape, C.PRISM18)
    N, dN = shape(ref)
    np.testing.assert_allclose(N, np.eye(len(ref)), atol=1e-15)
    pts = np.random.default_rng(0).uniform(-0.6, 0.2, (30, 3))
    N, dN = shape(pts)
    np.testing.assert_allclose(N.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(dN.sum(1), 0.0, atol=1e-14)
    f = lambda q: 1 + q[:, 0] ** 2 - 2 * q[:, 1] * q[:, 2] + 0.3 * q[:, 2] ** 2 + q[:, 0]   # noqa: E731
    np.testing.assert_allclose(N @ f(ref), f(pts), atol=1e-14)
    # derivative of f: (2x + 1, -2z, -2y + 0.6z)
    g = np.stack([2 * pts[:, 0] + 1, -2 * pts[:, 2], -2 * pts[:, 1] + 0.6 * pts[:, 2]], 1)
    np.testing.assert_allclose(np.einsum('ma,a->m', dN[:, :, 0], f(ref)), g[:, 0], atol=1e-13)
    np.testing.assert_allclose(np.einsum('ma,a->m', dN[:, :, 2], f(ref)), g[:, 2], atol=1e-13)


def _as_quadratic(d):
    """The same straight-sided mesh with 27/18 nodes: mid-edge/face/centre nodes at the linear
    map's positions, deduplicated by coordinates."""
    xyz = list(map(tuple, np.round(d.xyz, 12)))
    ids = {x: i for i, x in enumerate(xyz)}
    pts = list(d.xyz)

    def node(x):
        key = tuple(np.round(x, 12))
        if key not in ids:
            ids[key] = len(pts)
            pts.append(np.asarray(x))
        return ids[key]
    hexes = []
    for h in d.hex:
        X = d.xyz[h]
        out = []
        for c in C.HEX27:
            lam = np.array([np.prod([(1 + s[a] * c[a]) / 2 for a in range(3)]) for s in I.HEX_REF_VERTS])
            out.append(node(lam @ X))
        hexes.append(out)
    pris = []
    for pr in d.prism:
        X = d.xyz[pr]
        out = []
        for (r, s, z) in C.PRISM18:
            lam = np.array([-(r + s) / 2, (1 + r) / 2, (1 + s) / 2])
            w = np.concatenate([lam * (1 - z) / 2, lam * (1 + z) / 2])
            out.append(node(w @ X))
        pris.append(out)
    return I.MeshDesc(xyz=np.array(pts), hex=np.array(hexes, dtype=np.int64).reshape(-1, 27),
                      bface_nodes=d.bface_nodes, bface_tag=d.bface_tag, periodic=d.periodic, bcs=d.bcs,
                      prism=np.array(pris, dtype=np.int64).reshape(-1, 18))


@pytest.mark.parametrize("p", [2, 3])
def test_straight_sided_quadratic_equals_linear(p):
    d = I.hex_box_mesh((3, 3, 2), prisms="checker", seed=p, rotate=True, perturb=0.1)
    dq = _as_quadratic(d)
    m1, m2 = MixedFR(d, PH, p), MixedFR(dq, PH, p)
    for t in range(2):
        np.testing.assert_allclose(m2.S[t], m1.S[t], rtol=0, atol=1e-13)
        np.testing.assert_allclose(m2.detJ[t], m1.detJ[t], rtol=1e-13)
    Qs = [I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=1) for x in m1.x]
    for R1, R2 in zip(m1.residual(Qs), m2.residual(Qs)):
        np.testing.assert_allclose(R2, R1, rtol=0, atol=1e-12 * np.abs(R1).max())


def _flux_scale(m):
    """max|F| / h_min of the uniform state (rho = 1, u = (0.3, 0.2, 0.1), p = 1/gamma)."""
    U = [I.uniform_state(x.shape[:2]) for x in m.x]
    rho, u, pr = 1.0, np.array([0.3, 0.2, 0.1]), 1.0 / 1.4
    return (rho * u.max() ** 2 + pr) / min(h.min() for h in m.h if len(h)), U


@pytest.mark.parametrize("prisms", [None, "checker", "all"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_curved_free_stream_metric_identities_and_normals(prisms, p):
    d = I.curved_box_mesh((2, 2, 2), prisms=prisms, warp=0.15, seed=p, rotate=True, shuffle=True)
    m = MixedFR(d, PH, p)
    tol = 1e-13 * (p + 1) ** 2
    for t, S in zip(m.types, m.S):
        if len(S):
            ident = sum(np.einsum('mn,enj->emj', t.Dop[dd], S[:, :, dd, :]) for dd in range(3))
            assert np.abs(ident).max() <= tol * np.abs(S).max()
    mism = max(np.abs(m.nf[a][f][e] + m.nf[b][g][k][perm]).max() for (a, e, f, b, k, g, perm) in m.ifaces)
    assert mism <= tol * 10
    scale, U = _flux_scale(m)
    R = m.residual(U)
    assert max(np.abs(r).max() for r in R if r.size) <= tol * scale


@pytest.mark.parametrize("p", [2, 4])
def test_curved_conservation_and_orientation_invariance(p):
    ma = MixedFR(I.curved_box_mesh((3, 2, 2), prisms="checker", warp=0.12, seed=1), PH, p)
    mb = MixedFR(I.curved_box_mesh((3, 2, 2), prisms="checker", warp=0.12, seed=9, rotate=True, shuffle=True), PH, p)
    Qa = [I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=3) for x in ma.x]
    Ra = ma.residual(Qa)
    s = np.abs(ma.integrate(Ra))
    a = sum(np.einsum('m,em,emv->v', t.W, dJ, np.abs(r)) for t, dJ, r in zip(ma.types, ma.detJ, Ra))
    assert np.all(s <= 1e-12 * a)
    Qb = [I.tgv_state(x, Ma=0.2, perturb=1e-2, seed=3) for x in mb.x]
    Rb = mb.residual(Qb)
    for t in range(2):
        if ma.x[t].size == 0:
            continue
        ei = cKDTree(mb.x[t].mean(axis=1)).query(ma.x[t].mean(axis=1))[1]
        for e in range(ma.x[t].shape[0]):
            dd, i = cKDTree(mb.x[t][ei[e]]).query(ma.x[t][e])
            assert dd.max() < 1e-9
            np.testing.assert_allclose(Rb[t][ei[e]][i], Ra[t][e], rtol=0, atol=1e-11 * np.abs(Ra[t]).max())


@pytest.mark.parametrize("kind", ["hex", "prism"])
def test_curl_metrics_converge_to_analytic(kind):
    """On a general quadratic element the curl metrics equal the analytic adjugate once the
    interpolant is exact for the products X_l d_k X_m (degree <= 4), and differ below that."""
    shape, ref_nodes = (C.hex27_shape, C.HEX27) if kind == "hex" else (C.prism18_shape, C.PRISM18)
    q = ref_nodes.astype(np.float64)
    X = (q + 0.15 * np.stack([np.sin(q[:, 1] + 0.5 * q[:, 2]), np.cos(q[:, 0] * q[:, 2]),
                              0.5 * np.sin(q[:, 0] + q[:, 1])], 1))[None]
    ref = np.random.default_rng(1).uniform(-0.8, 0.0, (40, 3))
    _, dN = shape(ref)
    J = np.einsum('mab,eai->emib', dN, X)
    Sa = np.linalg.det(J)[..., None, None] * np.linalg.inv(J)
    errs = [np.abs(C.curved_geometry(kind, p)(X, ref)[2] - Sa).max() for p in (2, 3, 4, 6)]
    # below p = 4 the interpolant of the degree-4 products X_l d_k X_m is inexact ...
    assert errs[0] > 1e-2 and 1e-5 < errs[1] < 1e-2 * errs[0]
    # ... from p = 4 on it is exact, and the curl form returns the analytic adjugate.
    assert errs[2] < 1e-13 and errs[3] < 1e-13
