"""The library's host mesh build (fr_mesh_inspect: connectivity, solution points, metric terms;
no device work) against the oracles' independent geometry on the CPU: trilinear hexahedra
(rotated, shuffled, perturbed), prisms, and quadratic elements with curl-form metrics
(Eq. 1: S = |J| J^-1 and 1/|J| at the solution points)."""
import os

import numpy as np
import pytest

from oracle.hexfr import HexFR
from oracle.mixedfr import MixedFR
from paper_2308_06605_gb300 import build as B
from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not os.path.exists(fr.LIB_PATH):
        B.build()
    fr.load()


def _split_metrics(met, n_pts):
    S = met[:, :9, :].transpose(0, 2, 1).reshape(met.shape[0], n_pts, 3, 3)
    return S, met[:, 9, :]


@pytest.mark.parametrize("p", [1, 3, 5, 7])
def test_hexahedra_points_and_metrics(p):
    d = I.hex_box_mesh((3, 3, 2), seed=p, rotate=True, shuffle=True, perturb=0.12)
    r = fr.inspect(d, p)
    m = HexFR(d, I.tgv_physics(), p)
    assert r["n_elem"] == 18 and r["n_iface"] == 3 * 18 and r["n_bface"] == 0
    np.testing.assert_allclose(r["x"].reshape(m.x.shape), m.x, rtol=0, atol=1e-13)
    S, invJ = _split_metrics(r["metrics_hex"], r["n_pts"])
    np.testing.assert_allclose(S, m.S, rtol=0, atol=1e-13 * np.abs(m.S).max())
    np.testing.assert_allclose(invJ, 1.0 / m.detJ, rtol=1e-13)


@pytest.mark.parametrize("curved", [False, True])
@pytest.mark.parametrize("prisms", ["all", "checker"])
def test_mixed_and_curved_points_and_metrics(prisms, curved):
    p = 3
    d = (I.curved_box_mesh((2, 2, 2), prisms=prisms, warp=0.12, seed=4, rotate=True, shuffle=True) if curved else
         I.hex_box_mesh((3, 2, 2), prisms=prisms, seed=4, rotate=True, shuffle=True, perturb=0.1))
    r = fr.inspect(d, p)
    ora = MixedFR(d, I.tgv_physics(), p)
    x = np.concatenate([a.reshape(-1, 3) for a in ora.x])
    np.testing.assert_allclose(r["x"], x, rtol=0, atol=1e-13 * np.abs(x).max())
    for met, n_pts, S_o, J_o in ((r["metrics_hex"], r["n_pts"], ora.S[0], ora.detJ[0]),
                                 (r["metrics_prism"], r["n_pts_prism"], ora.S[1], ora.detJ[1])):
        if len(met) == 0:
            continue
        S, invJ = _split_metrics(met, n_pts)
        np.testing.assert_allclose(S, S_o, rtol=0, atol=1e-12 * np.abs(S_o).max())
        np.testing.assert_allclose(invJ, 1.0 / J_o, rtol=1e-12)


def test_walled_box_counts():
    d = I.hex_box_mesh((3, 2, 2), periodic=(False, True, True),
                       wall_tags={1: (I.BC_WALL_ISOTHERMAL, (1.0,)), 2: (I.BC_CHAR_OUTFLOW, (1.0,))})
    r = fr.inspect(d, 2)
    # interior + periodic interfaces: x-direction 2 x (2 x 2), y and z periodic 3 x 2 x 2 each
    assert r["n_iface"] == 8 + 12 + 12 and r["n_bface"] == 8


def test_inspect_reports_mesh_errors():
    d = I.hex_box_mesh((2, 2, 2))
    d.periodic[0].t = (1.0, 0.0, 0.0)
    with pytest.raises(fr.FRError, match="FR_EMESH"):
        fr.inspect(d, 2)
    with pytest.raises(fr.FRError, match="FR_EINVAL"):
        fr.inspect(I.hex_box_mesh((2, 2, 2)), 0)


def _slot(code, a, b, N):
    if code & 4:
        a, b = b, a
    if code & 1:
        a = N - 1 - a
    if code & 2:
        b = N - 1 - b
    return a + N * b


@pytest.mark.parametrize("p", [2, 4])
def test_face_table_orientation_and_normals(p):
    """Every element face point maps through the library's face table and orientation code to an
    interface slot where (i) the stored side-0 normal equals the oracle's outward area-scaled
    normal of that face point, negated on side 1, and (ii) both sides' oracle flux points
    coincide (modulo the periodic translation); every slot of every interface is used once per
    side."""
    N, Nf = p + 1, (p + 1) ** 2
    L = 2 * np.pi
    d = I.hex_box_mesh((3, 3, 2), seed=10 + p, rotate=True, shuffle=True, perturb=0.1)
    r = fr.inspect(d, p)
    ora = HexFR(d, I.tgv_physics(), p)
    n_if = r["n_iface"] + r["n_bface"]
    seen = {}
    for e in range(r["n_elem"]):
        for f in range(6):
            packed = int(r["ef"][e, f])
            iface, side, code = packed >> 4, (packed >> 3) & 1, packed & 7
            assert 0 <= iface < n_if
            for q in range(Nf):
                s = _slot(code, q % N, q // N, N)
                want = ora.nf[e, f, q] * (1.0 if side == 0 else -1.0)
                np.testing.assert_allclose(r["normals"][iface, :3, s], want, rtol=0, atol=1e-13)
                assert abs(r["normals"][iface, 3, s] - np.linalg.norm(want)) <= 1e-13
                key = (iface, s, side)
                assert key not in seen
                seen[key] = ora.xf[e, f, q]
    for iface in range(r["n_iface"]):
        for s in range(Nf):
            dx = seen[(iface, s, 0)] - seen[(iface, s, 1)]
            dx -= L * np.round(dx / L)
            assert np.abs(dx).max() <= 1e-12
    assert len(seen) == 2 * r["n_iface"] * Nf


@pytest.mark.parametrize("curved", [False, True])
@pytest.mark.parametrize("prisms", ["all", "checker"])
def test_mixed_face_tables_orientation_and_normals(prisms, curved):
    """As above on meshes with prisms (triangular faces through the triangle slot map, the
    quadrilateral faces of prisms through the same orientation codes as hexahedra), straight and
    curved, against the mixed-element oracle's face geometry."""
    p = 3
    N, Nf, Nt = p + 1, (p + 1) ** 2, (p + 1) * (p + 2) // 2
    L = 2 * np.pi
    d = (I.curved_box_mesh((2, 2, 2), prisms=prisms, warp=0.1, seed=6, rotate=True, shuffle=True) if curved else
         I.hex_box_mesh((3, 2, 2), prisms=prisms, seed=6, rotate=True, shuffle=True, perturb=0.1))
    r = fr.inspect(d, p)
    ora = MixedFR(d, I.tgv_physics(), p)
    seen = {}
    tables = [(0, r["ef"], 6), (1, r["ef_prism"], 5)]
    for t, ef, nfaces in tables:
        for e in range(ef.shape[0]):
            for f in range(nfaces):
                packed = int(ef[e, f])
                iface, side, code = packed >> 4, (packed >> 3) & 1, packed & 7
                tri = t == 1 and f < 2
                for q in range(Nt if tri else Nf):
                    s = int(r["tri_slot"][code, q]) if tri else _slot(code, q % N, q // N, N)
                    want = ora.nf[t][f][e][q] * (1.0 if side == 0 else -1.0)
                    np.testing.assert_allclose(r["normals"][iface, :3, s], want, rtol=0,
                                               atol=1e-12 * np.abs(want).max())
                    key = (iface, s, side)
                    assert key not in seen
                    seen[key] = ora.xf[t][f][e][q]
    pairs = 0
    for (iface, s, side), x0 in seen.items():
        if side == 0 and iface < r["n_iface"]:
            dx = x0 - seen[(iface, s, 1)]
            dx -= L * np.round(dx / L)
            assert np.abs(dx).max() <= 1e-12
            pairs += 1
    assert pairs * 2 == sum(1 for k in seen if k[0] < r["n_iface"])
