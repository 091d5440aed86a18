"""The C-ABI library builds, loads and exports every symbol its headers declare; host-side
validation runs before any device work (CPU only, no compute calls)."""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

from paper_2308_06605_gb300 import build as B
from paper_2308_06605_gb300 import fr, inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(fr.LIB_PATH):
        B.build()
    return fr.load()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(fr\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"fr_mesh_create", "fr_set_state", "fr_residual", "fr_rk_stage", "fr_free"} <= names
    for n in names:
        assert hasattr(lib, n), n


def _create(desc, phys, p, vcjh_c=0.0):
    lib = fr.load()
    xyz = np.ascontiguousarray(desc.xyz)
    hexa = np.ascontiguousarray(desc.hex)
    pri = np.ascontiguousarray(desc.prism if getattr(desc, "prism", None) is not None else np.zeros((0, 6), np.int64))
    bn = np.ascontiguousarray(desc.bface_nodes)
    bt = np.ascontiguousarray(desc.bface_tag)
    per = (fr.fr_periodic * max(1, len(desc.periodic)))()
    for i, pp in enumerate(desc.periodic):
        per[i].tag_a, per[i].tag_b = pp.tag_a, pp.tag_b
        for k in range(3):
            per[i].t[k] = pp.t[k]
    d = fr.fr_mesh_desc(n_nodes=xyz.shape[0], xyz=fr._ptr(xyz, C.c_double), n_hex=hexa.shape[0],
                        hex=fr._ptr(hexa, C.c_int64), p=p, n_bface=bn.shape[0],
                        bface_nodes=fr._ptr(bn, C.c_int64), bface_tag=fr._ptr(bt, C.c_int32),
                        n_bc=0, bc=None, n_periodic=len(desc.periodic), periodic=per,
                        n_prism=pri.shape[0], prism=fr._ptr(pri, C.c_int64))
    ph = fr.fr_physics(gamma=phys.gamma, R=phys.R, mu=phys.mu, Pr=phys.Pr, inviscid=0, viscous=phys.viscous,
                       br2_eta=6.0, precision=0, vcjh_c=vcjh_c)
    h = C.c_void_p()
    st = lib.fr_mesh_create(C.byref(d), C.byref(ph), 0, C.byref(h))
    return st, lib.fr_last_error(None).decode()


def test_invalid_order_rejected_before_device_work(lib):
    d = I.hex_box_mesh((2, 2, 2))
    for p in (0, 8, -1):
        st, msg = _create(d, I.tgv_physics(), p)
        assert st == fr.FR_EINVAL and "p must be" in msg


def test_bad_physics_rejected(lib):
    d = I.hex_box_mesh((2, 2, 2))
    ph = I.tgv_physics()
    ph.gamma = 1.0
    st, _ = _create(d, ph, 2)
    assert st == fr.FR_EINVAL


def test_unmatched_periodic_face_is_mesh_error(lib):
    d = I.hex_box_mesh((2, 2, 2))
    d.periodic[0].t = (1.0, 0.0, 0.0)          # wrong translation: x-faces find no partner
    st, msg = _create(d, I.tgv_physics(), 2)
    assert st == fr.FR_EMESH and "partner" in msg


def test_untagged_boundary_face_is_mesh_error(lib):
    d = I.hex_box_mesh((2, 2, 2))
    keep = d.bface_tag != 1
    d.bface_nodes, d.bface_tag = d.bface_nodes[keep], d.bface_tag[keep]
    st, msg = _create(d, I.tgv_physics(), 2)
    assert st == fr.FR_EMESH and "boundary tag" in msg


def test_inverted_element_is_mesh_error(lib):
    d = I.hex_box_mesh((2, 2, 2))
    d.hex[3] = d.hex[3][[4, 5, 6, 7, 0, 1, 2, 3]]   # mirrored: negative Jacobian
    st, msg = _create(d, I.tgv_physics(), 2)
    assert st == fr.FR_EMESH


def test_face_shared_by_three_elements_is_mesh_error(lib):
    d = I.hex_box_mesh((2, 2, 2))
    d.hex = np.concatenate([d.hex, d.hex[:1]])
    st, msg = _create(d, I.tgv_physics(), 2)
    assert st == fr.FR_EMESH and "shared by" in msg


def test_correction_parameter_checked_before_device_work(lib):
    """c must keep 1 + eta > 0 (eta = c (2p+1) (a_p p!)^2 / 2; at p = 2, a_p p! = 3, so the
    limit is c_- = -2/45); c != 0 is refused on meshes with prisms."""
    d = I.hex_box_mesh((2, 2, 2))
    for c in (-2.0 / 45.0 * 1.000001, -1.0, float("nan"), float("inf")):
        st, msg = _create(d, I.tgv_physics(), 2, vcjh_c=c)
        assert st == fr.FR_EINVAL and "correction parameter" in msg, (c, msg)
    st, msg = _create(I.hex_box_mesh((2, 2, 2), prisms="checker"), I.tgv_physics(), 2, vcjh_c=0.01)
    assert st == fr.FR_EUNSUPPORTED and "hexahedral" in msg


def test_per_element_orders_uniform_only(lib):
    """fr_mesh_desc.elem_p: uniform orders are accepted, an order outside 1..7 is FR_EINVAL and
    differing orders are FR_EUNSUPPORTED, all decided on the host before any device work."""
    d = I.hex_box_mesh((2, 2, 2))
    n = 8
    info = fr.inspect(d, 3, elem_p=np.full(n, 3, np.int8))
    assert info["n_elem"] == n
    ep = np.full(n, 3, np.int8)
    ep[5] = 4
    for call in (lambda: fr.inspect(d, 3, elem_p=ep), lambda: fr.Mesh(d, I.tgv_physics(), 3, elem_p=ep)):
        with pytest.raises(fr.FRError) as ei:
            call()
        assert ei.value.status == fr.FR_EUNSUPPORTED and "elem_p[5] = 4" in str(ei.value)
    ep[5] = 9
    with pytest.raises(fr.FRError) as ei:
        fr.inspect(d, 3, elem_p=ep)
    assert ei.value.status == fr.FR_EINVAL and "outside 1..7" in str(ei.value)
    with pytest.raises(ValueError):
        fr.inspect(d, 3, elem_p=np.full(n - 1, 3, np.int8))
