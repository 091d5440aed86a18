"""Thin ctypes binding of the C ABI in include/fr.h (argument marshalling only).

Every computation happens in the CUDA library `lib/libfr.so`; this module converts NumPy / torch
arguments into pointers and sizes and turns non-OK statuses into exceptions.  It never computes
a residual itself and has no CPU fallback: `load()` raises if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .inputs import MeshDesc, Physics

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libfr.so")

FR_OK, FR_EINVAL, FR_ENOMEM, FR_ECUDA, FR_EMESH, FR_EUNSUPPORTED, FR_ENONFINITE, FR_ETIMEOUT = range(8)
STATUS_NAMES = ["FR_OK", "FR_EINVAL", "FR_ENOMEM", "FR_ECUDA", "FR_EMESH", "FR_EUNSUPPORTED",
                "FR_ENONFINITE", "FR_ETIMEOUT"]
FR_HOST, FR_DEVICE = 0, 1
FR_RK44, FR_SSPRK33, FR_SSPRK104 = 0, 1, 2
FR_RESIDUAL_ONLY = -1
FR_PREC_FP64, FR_PREC_MIXED, FR_PREC_MIXED_TC, FR_PREC_MIXED_VF32 = 0, 1, 2, 3
RK_STAGES = {FR_RK44: 4, FR_SSPRK33: 3, FR_SSPRK104: 10}


class FRError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {message}")


class fr_bc(C.Structure):
    _fields_ = [("tag", C.c_int32), ("kind", C.c_int32), ("params", C.c_double * 8)]


class fr_periodic(C.Structure):
    _fields_ = [("tag_a", C.c_int32), ("tag_b", C.c_int32), ("t", C.c_double * 3)]


class fr_mesh_desc(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("xyz", C.POINTER(C.c_double)),
                ("n_hex", C.c_int64), ("hex", C.POINTER(C.c_int64)),
                ("p", C.c_int32),
                ("n_bface", C.c_int64), ("bface_nodes", C.POINTER(C.c_int64)),
                ("bface_tag", C.POINTER(C.c_int32)),
                ("n_bc", C.c_int32), ("bc", C.POINTER(fr_bc)),
                ("n_periodic", C.c_int32), ("periodic", C.POINTER(fr_periodic)),
                ("n_prism", C.c_int64), ("prism", C.POINTER(C.c_int64)),
                ("hex_nodes", C.c_int32), ("prism_nodes", C.c_int32),
                ("elem_p", C.POINTER(C.c_int8))]


class fr_physics(C.Structure):
    _fields_ = [("gamma", C.c_double), ("R", C.c_double), ("mu", C.c_double), ("Pr", C.c_double),
                ("inviscid", C.c_int32), ("viscous", C.c_int32), ("br2_eta", C.c_double),
                ("precision", C.c_int32), ("ldg_tau", C.c_double), ("vcjh_c", C.c_double)]


class fr_batch_info(C.Structure):
    _fields_ = [("n_cases", C.c_int32), ("block", C.c_int32), ("grid", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("n_points", C.c_int64), ("smem_bytes", C.c_int64), ("n_tasks", C.c_int32), ("mode", C.c_int32)]


class fr_mesh_info(C.Structure):
    _fields_ = [("n_elem", C.c_int64), ("p", C.c_int32), ("n_pts", C.c_int32),
                ("n_iface", C.c_int64), ("n_bface", C.c_int64), ("device_bytes", C.c_int64),
                ("n_prism", C.c_int64), ("n_pts_prism", C.c_int32), ("n_points", C.c_int64),
                ("device", C.c_int32)]


class fr_part_info(C.Structure):
    _fields_ = [("n_elem", C.c_int64), ("n_iface", C.c_int64), ("n_bface", C.c_int64), ("n_peers", C.c_int32),
                ("n_halo", C.c_int64)]


# Exported functions: name -> (restype, argtypes)
SIGNATURES = {
    "fr_mesh_create": (C.c_int, [C.POINTER(fr_mesh_desc), C.POINTER(fr_physics), C.c_size_t, C.POINTER(C.c_void_p)]),
    "fr_mesh_query": (C.c_int, [C.c_void_p, C.POINTER(fr_mesh_info)]),
    "fr_solution_points": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fr_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "fr_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "fr_residual": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_int32]),
    "fr_rk_stage": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_double, C.c_double]),
    "fr_max_dt": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_double)]),
    "fr_residual_static": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "fr_set_closure": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int32]),
    "fr_closure_nu": (C.c_int, [C.c_void_p, C.POINTER(C.c_float)]),
    "fr_set_source": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fr_project_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fr_mlp_workspace_floats": (C.c_int64, [C.c_int64]),
    "fr_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_size_t]),
    "fr_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_size_t]),
    "fr_mlp_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float, C.c_float, C.c_float,
                              C.c_float, C.c_int32, C.c_size_t]),
    "fr_profile": (C.c_int, [C.c_void_p, C.c_int32]),
    "fr_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.c_int32]),
    "fr_probe_fma": (C.c_int32, [C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
    "fr_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    "fr_batch_set_dt": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "fr_batch_rk_stage": (C.c_int, [C.c_void_p, C.c_int32, C.c_double]),
    "fr_batch_tune": (C.c_int, [C.c_void_p]),
    "fr_batch_query": (C.c_int, [C.c_void_p, C.POINTER(fr_batch_info)]),
    "fr_batch_debug": (C.c_int, [C.c_void_p, C.c_int32, C.c_int64]),
    "fr_batch_select": (C.c_int, [C.c_void_p, C.c_int32]),
    "fr_batch_free": (None, [C.c_void_p]),
    "fr_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "fr_partition": (C.c_int, [C.POINTER(fr_mesh_desc), C.c_int32, C.c_void_p]),
    "fr_partition_cost": (C.c_int, [C.POINTER(fr_mesh_desc), C.c_int32, C.c_double, C.c_double, C.c_void_p]),
    "fr_part_inspect": (C.c_int, [C.POINTER(fr_mesh_desc), C.c_void_p, C.c_int32, C.POINTER(fr_part_info),
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "fr_mesh_create_part": (C.c_int, [C.POINTER(fr_mesh_desc), C.POINTER(fr_physics), C.c_void_p, C.c_int32,
                                      C.c_size_t, C.POINTER(C.c_void_p)]),
    "fr_halo_query": (C.c_int, [C.c_void_p, C.POINTER(fr_part_info), C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p]),
    "fr_part_phase": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_void_p,
                                C.c_void_p, C.c_void_p]),
    "fr_free": (None, [C.c_void_p]),
    "fr_last_error": (C.c_char_p, [C.c_void_p]),
    "fr_basis_1d": (C.c_int, [C.c_int32, C.c_double] + [C.POINTER(C.c_double)] * 7),
    "fr_tri_basis": (C.c_int, [C.c_int32] + [C.POINTER(C.c_double)] * 4),
    "fr_transfer_matrix": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
    "fr_mesh_inspect": (C.c_int, [C.c_void_p] * 8),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libfr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise FileNotFoundError(f"{path} not built: run `python -m paper_2308_06605_gb300.build`")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _data_ptr(x):
    """(pointer, where) for a NumPy array (host) or a torch tensor (host or CUDA)."""
    if isinstance(x, np.ndarray):
        if not (x.flags["C_CONTIGUOUS"] and x.dtype == np.float64):
            raise ValueError("state arrays must be C-contiguous float64")
        return C.c_void_p(x.ctypes.data), FR_HOST
    if not (x.is_contiguous() and str(x.dtype) == "torch.float64"):
        raise ValueError("state tensors must be contiguous float64")
    return C.c_void_p(x.data_ptr()), (FR_DEVICE if x.is_cuda else FR_HOST)


def basis_1d(p: int, c: float = 0.0) -> dict:
    """fr_basis_1d: the library's 1D tables of order p (host computation, no device work)."""
    lib = load()
    N = p + 1
    out = {k: np.zeros(N * N if k == "D" else N) for k in ("x", "w", "D", "lm", "lp", "hm", "hp")}
    st = lib.fr_basis_1d(p, c, *[_ptr(out[k], C.c_double) for k in ("x", "w", "D", "lm", "lp", "hm", "hp")])
    if st != FR_OK:
        raise FRError(st, "fr_basis_1d: order or correction parameter out of range")
    out["D"] = out["D"].reshape(N, N)
    return out


def tri_basis(p: int) -> dict:
    """fr_tri_basis: the library's triangle tables of order p (host computation)."""
    lib = load()
    Nt = (p + 1) * (p + 2) // 2
    out = {"rs": np.zeros((Nt, 2)), "Dr": np.zeros((Nt, Nt)), "Ds": np.zeros((Nt, Nt)), "Minv": np.zeros((Nt, Nt))}
    st = lib.fr_tri_basis(p, *[_ptr(out[k], C.c_double) for k in ("rs", "Dr", "Ds", "Minv")])
    if st != FR_OK:
        raise FRError(st, "fr_tri_basis: order out of range")
    return out


def transfer_matrix(kind: int, p: int, q: int) -> np.ndarray:
    """fr_transfer_matrix: the order-p -> order-q projection operator (0 line, 1 triangle)."""
    lib = load()
    n = (lambda k: k + 1) if kind == 0 else (lambda k: (k + 1) * (k + 2) // 2)
    T = np.zeros((n(q), n(p)))
    st = lib.fr_transfer_matrix(kind, p, q, _ptr(T, C.c_double))
    if st != FR_OK:
        raise FRError(st, "fr_transfer_matrix: bad kind or order")
    return T


def probe_fma(precision: int = 0, iters: int = 20000) -> float:
    """Measured FMA throughput of the current device in FLOP/s (0 = FP64, 1 = FP32)."""
    lib = load()
    v = C.c_double()
    if lib.fr_probe_fma(precision, iters, C.byref(v)) != 0:
        raise RuntimeError("fr_probe_fma failed")
    return v.value


def _describe(desc: MeshDesc, p: int, elem_p=None):
    """The C mesh description of `desc` at order p, and the arrays it points into (keep alive).
    elem_p: optional per-element orders (hexahedra first); the library builds uniform orders only."""
    xyz = np.ascontiguousarray(desc.xyz, dtype=np.float64)
    hexa = np.asarray(desc.hex, dtype=np.int64)
    hexa = np.ascontiguousarray(hexa if hexa.ndim == 2 else hexa.reshape(-1, 8))    # 8 or 27 nodes each
    pri = getattr(desc, "prism", None)
    pri = np.asarray(np.zeros((0, 6)) if pri is None else pri, dtype=np.int64)
    pri = np.ascontiguousarray(pri if pri.ndim == 2 else pri.reshape(-1, 6))           # 6 or 18 nodes each
    bn = np.ascontiguousarray(desc.bface_nodes, dtype=np.int64).reshape(-1, 4)
    bt = np.ascontiguousarray(desc.bface_tag, dtype=np.int32)
    bcs = (fr_bc * max(1, len(desc.bcs)))()
    for i, bc in enumerate(desc.bcs):
        bcs[i].tag, bcs[i].kind = bc.tag, bc.kind
        for k, v in enumerate(bc.params[:8]):
            bcs[i].params[k] = v
    per = (fr_periodic * max(1, len(desc.periodic)))()
    for i, pp in enumerate(desc.periodic):
        per[i].tag_a, per[i].tag_b = pp.tag_a, pp.tag_b
        for k in range(3):
            per[i].t[k] = pp.t[k]
    d = fr_mesh_desc(n_nodes=xyz.shape[0], xyz=_ptr(xyz, C.c_double), n_hex=hexa.shape[0],
                     hex=_ptr(hexa, C.c_int64), p=p, n_bface=bn.shape[0],
                     bface_nodes=_ptr(bn, C.c_int64), bface_tag=_ptr(bt, C.c_int32),
                     n_bc=len(desc.bcs), bc=bcs, n_periodic=len(desc.periodic), periodic=per,
                     n_prism=pri.shape[0], prism=_ptr(pri, C.c_int64),
                     hex_nodes=hexa.shape[1], prism_nodes=pri.shape[1])
    keep = [xyz, hexa, pri, bn, bt, bcs, per]
    if elem_p is not None:
        ep = np.ascontiguousarray(elem_p, dtype=np.int8)
        if ep.size != hexa.shape[0] + pri.shape[0]:
            raise ValueError(f"elem_p has {ep.size} entries, the mesh has {hexa.shape[0] + pri.shape[0]} elements")
        d.elem_p = _ptr(ep, C.c_int8)
        keep.append(ep)
    return d, keep


def inspect(desc: MeshDesc, p: int, elem_p=None) -> dict:
    """fr_mesh_inspect: sizes, solution points, metric terms, face table and interface normals of
    the host mesh build (no device work).  Points are [n_points][3]; metrics split into hexahedra
    [n_elem][10][n_pts] and prisms [n_prism][10][n_pts_prism]; ef [n_elem][6]; normals
    [n_iface + n_bface][4][(p+1)^2]."""
    lib = load()
    d, keep = _describe(desc, p, elem_p)
    info = fr_mesh_info()
    st = lib.fr_mesh_inspect(C.byref(d), C.byref(info), None, None, None, None, None, None)
    if st != FR_OK:
        raise FRError(st, lib.fr_last_error(None).decode())
    x = np.zeros((info.n_points, 3))
    nh, nph = info.n_elem * 10 * info.n_pts, info.n_prism * 10 * info.n_pts_prism
    met = np.zeros(nh + nph)
    Nf = (p + 1) ** 2
    ef = np.zeros((info.n_elem, 6), dtype=np.int32)
    nrm = np.zeros((info.n_iface + info.n_bface, 4, Nf))
    ef_p = np.zeros((info.n_prism, 5), dtype=np.int32)
    tri_slot = np.zeros((6, (p + 1) * (p + 2) // 2), dtype=np.int32)
    st = lib.fr_mesh_inspect(C.byref(d), C.byref(info), C.c_void_p(x.ctypes.data), C.c_void_p(met.ctypes.data),
                             C.c_void_p(ef.ctypes.data), C.c_void_p(nrm.ctypes.data),
                             C.c_void_p(ef_p.ctypes.data), C.c_void_p(tri_slot.ctypes.data))
    if st != FR_OK:
        raise FRError(st, lib.fr_last_error(None).decode())
    del keep
    return {"n_elem": info.n_elem, "n_pts": info.n_pts, "n_iface": info.n_iface, "n_bface": info.n_bface,
            "n_prism": info.n_prism, "n_pts_prism": info.n_pts_prism, "n_points": info.n_points, "x": x,
            "metrics_hex": met[:nh].reshape(info.n_elem, 10, info.n_pts),
            "metrics_prism": met[nh:].reshape(info.n_prism, 10, info.n_pts_prism), "ef": ef, "normals": nrm,
            "ef_prism": ef_p, "tri_slot": tri_slot}


def _physics(phys: Physics) -> fr_physics:
    return fr_physics(gamma=phys.gamma, R=phys.R, mu=phys.mu, Pr=phys.Pr, inviscid=phys.inviscid_flux,
                      viscous=phys.viscous, br2_eta=phys.br2_eta, precision=phys.precision,
                      ldg_tau=getattr(phys, "ldg_tau", 0.1), vcjh_c=getattr(phys, "vcjh_c", 0.0))


class Mesh:
    """One FR discretisation living on the current CUDA device (owns the C-side fr_mesh).

    States and residuals are [n_elem][n_pts][5] on hexahedral meshes; on meshes with prisms they
    are [n_points][5], the hexahedral points first (see `split`).
    """

    def __init__(self, desc: MeshDesc, phys: Physics, p: int, stream: int = 0, elem_p=None):
        lib = load()
        self._lib = lib
        self._keep = []
        d, keep = _describe(desc, p, elem_p)
        self._keep += keep
        ph = _physics(phys)
        h = C.c_void_p()
        st = self._create(lib, d, ph, stream, h)
        if st != FR_OK:
            raise FRError(st, lib.fr_last_error(None).decode())
        self._h = h
        info = fr_mesh_info()
        lib.fr_mesh_query(h, C.byref(info))
        self.n_elem, self.p, self.n_pts = info.n_elem, info.p, info.n_pts
        self.n_iface, self.n_bface, self.device_bytes = info.n_iface, info.n_bface, info.device_bytes
        self.n_prism, self.n_pts_prism, self.n_points = info.n_prism, info.n_pts_prism, info.n_points
        self.shape = (self.n_elem, self.n_pts, 5) if self.n_prism == 0 else (self.n_points, 5)
        self.device = info.device

    def _create(self, lib, d, ph, stream, h):
        return lib.fr_mesh_create(C.byref(d), C.byref(ph), stream, C.byref(h))

    def _check(self, st):
        if st != FR_OK:
            raise FRError(st, self._lib.fr_last_error(self._h).decode())

    def solution_points(self) -> np.ndarray:
        x = np.empty(self.shape[:-1] + (3,))
        self._check(self._lib.fr_solution_points(self._h, C.c_void_p(x.ctypes.data)))
        return x

    def split(self, a):
        """Views of a [n_points][k] array as (hexahedra [n_elem][n_pts][k], prisms [n_prism][n_pts_prism][k])."""
        nh = self.n_elem * self.n_pts
        k = a.shape[-1]
        flat = a.reshape(-1, k)
        return flat[:nh].reshape(self.n_elem, self.n_pts, k), flat[nh:].reshape(self.n_prism, self.n_pts_prism, k)

    def set_state(self, Q):
        p, where = _data_ptr(Q)
        self._check(self._lib.fr_set_state(self._h, p, where))

    def get_state(self, out=None):
        if out is None:
            out = np.empty(self.shape)
        p, where = _data_ptr(out)
        self._check(self._lib.fr_get_state(self._h, p, where))
        return out

    def residual(self, t: float = 0.0, out=None):
        if out is None:
            out = np.empty(self.shape)
        p, where = _data_ptr(out)
        self._check(self._lib.fr_residual(self._h, t, p, where))
        return out

    def residual_static(self, Q_device, R_device):
        """fr_residual_static: residual of a device state into a device buffer, no allocation."""
        q, wq = _data_ptr(Q_device)
        r, wr = _data_ptr(R_device)
        if wq != FR_DEVICE or wr != FR_DEVICE:
            raise ValueError("fr_residual_static takes device tensors")
        n = int(np.prod(self.shape))
        for name, x in (("Q_device", Q_device), ("R_device", R_device)):
            if x.numel() != n:
                raise ValueError(f"fr_residual_static: {name} has {x.numel()} values, the mesh's state has {n}")
            if x.device.index != self.device:
                raise ValueError(f"fr_residual_static: {name} is on cuda:{x.device.index}, the mesh on cuda:{self.device}")
        self._check(self._lib.fr_residual_static(self._h, q, r))

    def rk_stage(self, stage: int, t: float, dt: float, scheme: int = FR_RK44):
        self._check(self._lib.fr_rk_stage(self._h, scheme, stage, t, dt))

    def rk_step(self, t: float, dt: float, scheme: int = FR_RK44):
        for s in range(RK_STAGES[scheme]):
            self.rk_stage(s, t, dt, scheme)

    def max_dt(self, cfl: float) -> float:
        v = C.c_double()
        self._check(self._lib.fr_max_dt(self._h, cfl, C.byref(v)))
        return v.value

    def set_closure(self, params, scales, enable: bool = True):
        """Eddy-viscosity network: params (9153 floats), scales (mean[11], std[11], s_out)."""
        p = np.ascontiguousarray(params, dtype=np.float32)
        sc = np.ascontiguousarray(scales, dtype=np.float32)
        self._keep_closure = (p, sc)
        self._check(self._lib.fr_set_closure(self._h, p.ctypes.data_as(C.POINTER(C.c_float)),
                                             sc.ctypes.data_as(C.POINTER(C.c_float)), 1 if enable else 0))

    def set_source(self, accel=None, sigma=None, Q_ref=None):
        """Source term: body acceleration (3,) and / or sponge strength sigma [n_points] with its
        reference state Q_ref [n_points][5] (canonical order); None switches a part off."""
        a = None if accel is None else np.ascontiguousarray(accel, dtype=np.float64)
        sg = None if sigma is None else np.ascontiguousarray(sigma, dtype=np.float64).ravel()
        qr = None if Q_ref is None else np.ascontiguousarray(Q_ref, dtype=np.float64)
        self._keep_source = (a, sg, qr)
        ptr = lambda x: None if x is None else C.c_void_p(x.ctypes.data)   # noqa: E731
        self._check(self._lib.fr_set_source(self._h, ptr(a), ptr(sg), ptr(qr)))

    def closure_nu(self):
        out = np.empty(self.n_elem, dtype=np.float32)
        self._check(self._lib.fr_closure_nu(self._h, out.ctypes.data_as(C.POINTER(C.c_float))))
        return out

    def profile(self, enable: bool):
        self._check(self._lib.fr_profile(self._h, 1 if enable else 0))

    def profile_read(self, n: int = 4):
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        self._check(self._lib.fr_profile_read(self._h, ms, cnt, n))
        return list(ms), list(cnt)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fr_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def partition(desc: MeshDesc, p: int, n_parts: int, cost=None) -> np.ndarray:
    """fr_partition: part id of every element (recursive coordinate bisection; host only),
    balancing solution points, or with cost = (per hexahedral point, per prism point) the work
    (fr_partition_cost)."""
    lib = load()
    d, keep = _describe(desc, p)
    part = np.zeros(d.n_hex + d.n_prism, dtype=np.int32)
    if cost is None:
        st = lib.fr_partition(C.byref(d), n_parts, C.c_void_p(part.ctypes.data))
    else:
        st = lib.fr_partition_cost(C.byref(d), n_parts, float(cost[0]), float(cost[1]), C.c_void_p(part.ctypes.data))
    if st != FR_OK:
        raise FRError(st, lib.fr_last_error(None).decode())
    del keep
    return part


def _halo_arrays(info):
    return (np.zeros(max(1, info.n_peers), np.int32), np.zeros(info.n_peers + 1, np.int64),
            np.zeros(max(1, info.n_halo), np.int64), np.zeros(info.n_elem, np.int64))


def _halo_dict(info, arrs):
    peers, begin, gid, eg = arrs
    return {"n_elem": info.n_elem, "n_iface": info.n_iface, "n_bface": info.n_bface, "n_peers": info.n_peers,
            "n_halo": info.n_halo, "peers": peers[:info.n_peers].copy(), "peer_begin": begin.copy(),
            "gid": gid[:info.n_halo].copy(), "elem_global": eg.copy()}


def part_inspect(desc: MeshDesc, p: int, part, rank: int) -> dict:
    """fr_part_inspect: sizes and halo lists of part `rank` (host only, no device work)."""
    lib = load()
    d, keep = _describe(desc, p)
    pa = np.ascontiguousarray(part, dtype=np.int32)
    info = fr_part_info()
    st = lib.fr_part_inspect(C.byref(d), C.c_void_p(pa.ctypes.data), rank, C.byref(info), None, None, None, None)
    if st != FR_OK:
        raise FRError(st, lib.fr_last_error(None).decode())
    arrs = _halo_arrays(info)
    st = lib.fr_part_inspect(C.byref(d), C.c_void_p(pa.ctypes.data), rank, C.byref(info),
                             *[C.c_void_p(a.ctypes.data) for a in arrs])
    if st != FR_OK:
        raise FRError(st, lib.fr_last_error(None).decode())
    del keep
    return _halo_dict(info, arrs)


class PartMesh(Mesh):
    """Part `rank` of a domain-decomposed hexahedral mesh (fr_mesh_create_part).  States are in
    the part's local element order: `halo()["elem_global"]` gives each local element's index in
    the whole mesh.  With halo interfaces, stages run through `phase` (three calls per stage with
    the caller moving halo entries between them)."""

    def __init__(self, desc: MeshDesc, phys: Physics, p: int, part, rank: int, stream: int = 0):
        self._part = np.ascontiguousarray(part, dtype=np.int32)
        self._rank = int(rank)
        super().__init__(desc, phys, p, stream)
        self._halo = self.halo()

    def _create(self, lib, d, ph, stream, h):
        return lib.fr_mesh_create_part(C.byref(d), C.byref(ph), C.c_void_p(self._part.ctypes.data), self._rank,
                                       stream, C.byref(h))

    def halo(self) -> dict:
        info = fr_part_info()
        self._check(self._lib.fr_halo_query(self._h, C.byref(info), None, None, None, None))
        arrs = _halo_arrays(info)
        self._check(self._lib.fr_halo_query(self._h, C.byref(info), *[C.c_void_p(a.ctypes.data) for a in arrs]))
        return _halo_dict(info, arrs)

    def phase(self, phase: int, scheme: int = FR_RESIDUAL_ONLY, stage: int = 0, t: float = 0.0, dt: float = 0.0,
              recv=None, send=None, R=None):
        """fr_part_phase with device tensors (recv, send: float64 of n_halo * nv * (p+1)^2 values)."""
        ptr = lambda x: None if x is None else C.c_void_p(x.data_ptr())        # noqa: E731
        self._check(self._lib.fr_part_phase(self._h, phase, scheme, stage, t, dt, ptr(recv), ptr(send), ptr(R)))


def project_state(src: "Mesh", dst: "Mesh"):
    """fr_project_state: dst's state = the L2 projection of src's state onto dst's order."""
    st = src._lib.fr_project_state(src._h, dst._h)
    if st != FR_OK:
        raise FRError(st, src._lib.fr_last_error(dst._h).decode())


class Batch:
    """Ensemble of meshes advanced together by one persistent launch per RK stage."""

    def __init__(self, meshes):
        lib = load()
        self._lib = lib
        self.meshes = list(meshes)          # keep the borrowed meshes alive
        arr = (C.c_void_p * len(self.meshes))(*[m._h.value for m in self.meshes])
        h = C.c_void_p()
        st = lib.fr_batch_create(arr, len(self.meshes), C.byref(h))
        if st != FR_OK:
            raise FRError(st, lib.fr_batch_last_error(None).decode())
        self._h = h

    def _check(self, st):
        if st != FR_OK:
            raise FRError(st, self._lib.fr_batch_last_error(self._h).decode())

    def set_dt(self, dts):
        a = np.ascontiguousarray(dts, dtype=np.float64)
        self._check(self._lib.fr_batch_set_dt(self._h, a.ctypes.data_as(C.POINTER(C.c_double))))

    def rk_stage(self, stage: int, t: float = 0.0):
        self._check(self._lib.fr_batch_rk_stage(self._h, stage, t))

    def rk_step(self, t: float = 0.0):
        for s in range(4):
            self.rk_stage(s, t)

    def tune(self):
        self._check(self._lib.fr_batch_tune(self._h))

    def info(self) -> dict:
        i = fr_batch_info()
        self._check(self._lib.fr_batch_query(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in fr_batch_info._fields_}

    def select(self, mode: int):
        self._check(self._lib.fr_batch_select(self._h, mode))

    def debug(self, skip_block: int, spin_limit: int):
        self._check(self._lib.fr_batch_debug(self._h, skip_block, spin_limit))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fr_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


N_CLOSURE_PARAMS = 9153


class MLPTrainer:
    """Device-side training of the closure network through fr_mlp_* (torch tensors for memory)."""

    def __init__(self, params, scales, max_batch: int, stream: int = 0):
        import torch
        self._lib = load()
        self.torch = torch
        self.stream = stream
        self.P = torch.as_tensor(np.asarray(params, dtype=np.float32)).cuda().contiguous()
        self.sc = torch.as_tensor(np.asarray(scales, dtype=np.float32)).cuda().contiguous()
        self.g = torch.zeros_like(self.P)
        self.m = torch.zeros_like(self.P)
        self.v = torch.zeros_like(self.P)
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.work = torch.empty(int(self._lib.fr_mlp_workspace_floats(max_batch)), dtype=torch.float32, device="cuda")
        self.max_batch = max_batch
        self.step_count = 0

    @staticmethod
    def _p(t):
        return C.c_void_p(t.data_ptr())

    def loss_grad(self, X, y):
        n = X.shape[0]
        assert n <= self.max_batch
        st = self._lib.fr_mlp_loss_grad(self._p(self.P), self._p(self.sc), self._p(X), self._p(y), n, self._p(self.g),
                                        self._p(self.loss), self._p(self.work), self.stream)
        if st != FR_OK:
            raise FRError(st, "fr_mlp_loss_grad")
        return self.loss, self.g

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_count += 1
        st = self._lib.fr_mlp_adam(self._p(self.P), self._p(self.g), self._p(self.m), self._p(self.v), self.P.numel(),
                                   lr, beta1, beta2, eps, self.step_count, self.stream)
        if st != FR_OK:
            raise FRError(st, "fr_mlp_adam")

    def forward(self, X):
        n = X.shape[0]
        assert n <= self.max_batch
        out = self.torch.empty(n, dtype=self.torch.float32, device="cuda")
        st = self._lib.fr_mlp_forward(self._p(self.P), self._p(self.sc), self._p(X), n, self._p(out), self._p(self.work),
                                      self.stream)
        if st != FR_OK:
            raise FRError(st, "fr_mlp_forward")
        return out
