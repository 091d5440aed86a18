"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds workload definitions only: hexahedral box meshes (with optional element
shuffling, random local vertex rotations and interior-node perturbation), boundary tags,
periodic pairings, and the initial-condition fields (Taylor-Green vortex, isentropic vortex,
uniform flow) as functions of physical coordinates.  It contains none of the flux-reconstruction
arithmetic: no basis, no operators, no fluxes.  Both the CUDA library and the oracle receive the
same arrays from here and build everything else on their own.

Vertex order of a hexahedron follows VTK/CGNS: bottom face (zeta=-1) counter-clockwise seen
from inside +zeta, then the top face in the same order.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

# Boundary-condition kinds (match the C enum in include/fr.h).
BC_WALL_ISOTHERMAL = 1      # no-slip isothermal wall, params[0] = T_wall
BC_CHAR_INFLOW = 2          # characteristic subsonic inflow, params = (p0, T0, nx, ny, nz)
BC_CHAR_OUTFLOW = 3         # characteristic subsonic outflow, params[0] = p_static
BC_DIRICHLET = 4            # exact-state ghost, params = (rho, rhou, rhov, rhow, E)

# Reference coordinates of the 8 hex vertices in VTK order.
HEX_REF_VERTS = np.array([
    [-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
    [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], dtype=np.int64)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n uint64 draws of the splitmix64 generator (Steele, Lea & Flood 2014) from `seed`."""
    out = np.empty(n, dtype=np.uint64)
    s = int(seed) & 0xFFFFFFFFFFFFFFFF
    for i in range(n):
        s = (s + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        out[i] = z ^ (z >> 31)
    return out


def splitmix64_uniform(seed: int, n: int) -> np.ndarray:
    """n doubles in [0,1) from the top 53 bits of splitmix64 draws."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


@dataclass
class BC:
    tag: int
    kind: int
    params: Tuple[float, ...] = ()


@dataclass
class Periodic:
    """Faces tagged `tag_b` are the faces tagged `tag_a` translated by `t`."""
    tag_a: int
    tag_b: int
    t: Tuple[float, float, float]


@dataclass
class MeshDesc:
    xyz: np.ndarray                     # [n_nodes][3] float64
    hex: np.ndarray                     # [E][8] int64 node ids, VTK order
    bface_nodes: np.ndarray             # [nb][4] int64 node ids of each boundary face (-1 pads a triangle)
    bface_tag: np.ndarray               # [nb] int32
    periodic: List[Periodic] = field(default_factory=list)
    bcs: List[BC] = field(default_factory=list)
    prism: np.ndarray = field(default_factory=lambda: np.zeros((0, 6), dtype=np.int64))   # [Ep][6] VTK order

    @property
    def n_elem(self) -> int:
        return int(self.hex.shape[0])


def cube_rotations() -> np.ndarray:
    """The 24 proper rotations of the cube as signed 3x3 permutation matrices (det = +1)."""
    mats = []
    for perm in [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]:
        for sx in (1, -1):
            for sy in (1, -1):
                for sz in (1, -1):
                    m = np.zeros((3, 3), dtype=np.int64)
                    for r, (c, s) in enumerate(zip(perm, (sx, sy, sz))):
                        m[r, c] = s
                    if round(np.linalg.det(m)) == 1:
                        mats.append(m)
    assert len(mats) == 24
    return np.array(mats)


def rotation_vertex_permutations() -> np.ndarray:
    """[24][8]: new local vertex k takes the old local vertex perm[r][k].

    Rotating the reference frame maps reference vertex k to R @ c_k; the element's shape is
    unchanged, only its local frame changes.
    """
    lookup = {tuple(v): i for i, v in enumerate(HEX_REF_VERTS.tolist())}
    perms = []
    for R in cube_rotations():
        perms.append([lookup[tuple((R @ c).tolist())] for c in HEX_REF_VERTS])
    return np.array(perms, dtype=np.int64)


# Proper relabelings of a prism's vertices (VTK order): the three rotations of the triangle and
# the three top/bottom exchanges combined with a reflection of the triangle.
PRISM_PERMUTATIONS = np.array([[0, 1, 2, 3, 4, 5], [1, 2, 0, 4, 5, 3], [2, 0, 1, 5, 3, 4],
                               [3, 5, 4, 0, 2, 1], [4, 3, 5, 1, 0, 2], [5, 4, 3, 2, 1, 0]], dtype=np.int64)


def hex_box_mesh(n: Sequence[int], lo=(0.0, 0.0, 0.0), hi=(2 * np.pi,) * 3,
                 periodic=(True, True, True), seed: int | None = None,
                 shuffle: bool = False, rotate: bool = False, perturb: float = 0.0,
                 wall_tags: dict | None = None, affine=None, prisms=None) -> MeshDesc:
    """Structured box of nx*ny*nz hexahedra stored as an unstructured mesh.

    Boundary faces are tagged 1..6 for x-, x+, y-, y+, z-, z+.  Periodic axes pair (1,2), (3,4),
    (5,6) with the box length as translation.  `perturb` moves interior nodes by a seeded
    uniform displacement of that fraction of the local spacing (straight-sided trilinear
    elements).  `shuffle` permutes the element order and `rotate` applies a random one of the
    24 cube rotations to each element's local vertex order; both are seeded.  `affine` (3x3)
    maps the box about `lo` (x -> lo + A (x - lo)), giving a sheared lattice of parallelepipeds;
    periodic translations are mapped with it.  `prisms` = "all" or "checker" splits every (or every
    other) column of hexahedra along z into two prisms each (cut through the diagonal from corner
    0 to corner 2 of every bottom face); z-boundary faces of split columns are triangles.
    """
    nx, ny, nz = (int(v) for v in n)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    rng = np.random.default_rng(seed if seed is not None else 0)
    xs = [np.linspace(lo[a], hi[a], m + 1) for a, m in enumerate((nx, ny, nz))]
    X, Y, Z = np.meshgrid(xs[0], xs[1], xs[2], indexing="ij")
    xyz = np.stack([X, Y, Z], axis=-1)            # [nx+1][ny+1][nz+1][3]
    if perturb > 0.0:
        h = (hi - lo) / np.array([nx, ny, nz])
        d = rng.uniform(-perturb, perturb, size=xyz.shape) * h
        interior = np.zeros(xyz.shape[:3], dtype=bool)
        interior[1:-1, 1:-1, 1:-1] = True
        xyz = xyz + d * interior[..., None]
    nid = np.arange((nx + 1) * (ny + 1) * (nz + 1)).reshape(nx + 1, ny + 1, nz + 1)
    xyz = xyz.reshape(-1, 3)
    A = np.eye(3) if affine is None else np.asarray(affine, dtype=np.float64)
    xyz = lo[None, :] + (xyz - lo[None, :]) @ A.T
    hexes = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                hexes.append([nid[i, j, k], nid[i + 1, j, k], nid[i + 1, j + 1, k], nid[i, j + 1, k],
                              nid[i, j, k + 1], nid[i + 1, j, k + 1], nid[i + 1, j + 1, k + 1],
                              nid[i, j + 1, k + 1]])
    hexes = np.array(hexes, dtype=np.int64)
    split = np.zeros((nx, ny), dtype=bool)
    if prisms == "all":
        split[:] = True
    elif prisms == "checker":
        split[(np.add.outer(np.arange(nx), np.arange(ny)) % 2) == 0] = True
    is_split = np.array([split[i, j] for k in range(nz) for j in range(ny) for i in range(nx)], dtype=bool)
    prism_list = []
    for hv in hexes[is_split]:
        prism_list.append([hv[0], hv[1], hv[2], hv[4], hv[5], hv[6]])
        prism_list.append([hv[0], hv[2], hv[3], hv[4], hv[6], hv[7]])
    prism_arr = np.array(prism_list, dtype=np.int64).reshape(-1, 6)
    hexes = hexes[~is_split]
    # Boundary quads with tags.
    bnodes, btags = [], []
    for j in range(ny):
        for k in range(nz):
            bnodes.append([nid[0, j, k], nid[0, j + 1, k], nid[0, j + 1, k + 1], nid[0, j, k + 1]]); btags.append(1)
            bnodes.append([nid[nx, j, k], nid[nx, j + 1, k], nid[nx, j + 1, k + 1], nid[nx, j, k + 1]]); btags.append(2)
    for i in range(nx):
        for k in range(nz):
            bnodes.append([nid[i, 0, k], nid[i + 1, 0, k], nid[i + 1, 0, k + 1], nid[i, 0, k + 1]]); btags.append(3)
            bnodes.append([nid[i, ny, k], nid[i + 1, ny, k], nid[i + 1, ny, k + 1], nid[i, ny, k + 1]]); btags.append(4)
    for i in range(nx):
        for j in range(ny):
            for kk, tag in ((0, 5), (nz, 6)):
                c = [nid[i, j, kk], nid[i + 1, j, kk], nid[i + 1, j + 1, kk], nid[i, j + 1, kk]]
                if split[i, j]:
                    bnodes.append([c[0], c[1], c[2], -1]); btags.append(tag)
                    bnodes.append([c[0], c[2], c[3], -1]); btags.append(tag)
                else:
                    bnodes.append(c); btags.append(tag)
    per = []
    L = hi - lo
    for a in range(3):
        if periodic[a]:
            t = np.zeros(3)
            t[a] = float(L[a])
            per.append(Periodic(2 * a + 1, 2 * a + 2, tuple(float(v) for v in A @ t)))
    bcs = []
    if wall_tags:
        for tag, (kind, params) in wall_tags.items():
            bcs.append(BC(int(tag), int(kind), tuple(float(v) for v in params)))
    if rotate:
        perms = rotation_vertex_permutations()
        r = rng.integers(0, 24, size=hexes.shape[0])
        hexes = np.take_along_axis(hexes, perms[r], axis=1)
        if len(prism_arr):
            r = rng.integers(0, 6, size=prism_arr.shape[0])
            prism_arr = np.take_along_axis(prism_arr, PRISM_PERMUTATIONS[r], axis=1)
    if shuffle:
        hexes = hexes[rng.permutation(hexes.shape[0])]
        prism_arr = prism_arr[rng.permutation(prism_arr.shape[0])]
    return MeshDesc(xyz=np.ascontiguousarray(xyz, dtype=np.float64),
                    hex=np.ascontiguousarray(hexes, dtype=np.int64),
                    bface_nodes=np.array(bnodes, dtype=np.int64).reshape(-1, 4),
                    bface_tag=np.array(btags, dtype=np.int32),
                    periodic=per, bcs=bcs, prism=np.ascontiguousarray(prism_arr, dtype=np.int64))


# ---------------------------------------------------------------------------------------------
# Quadratic (curved) elements.  Node orders (reference coordinates):
#   27-node hexahedron: the 8 corners (VTK order), the 12 edge midpoints (bottom 01 12 23 30, top
#   45 56 67 74, vertical 04 15 26 37), the 6 face centres (x-, x+, y-, y+, z-, z+), the centre.
#   18-node prism: the 6 corners (VTK wedge order), the edge midpoints 01 12 20 (bottom), 34 45 53
#   (top), 03 14 25 (vertical), then the centres of the quadrilateral faces 0143, 1254, 2035.
# ---------------------------------------------------------------------------------------------
HEX27_REF = np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1], [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1],
                      [0, -1, -1], [1, 0, -1], [0, 1, -1], [-1, 0, -1], [0, -1, 1], [1, 0, 1], [0, 1, 1], [-1, 0, 1],
                      [-1, -1, 0], [1, -1, 0], [1, 1, 0], [-1, 1, 0],
                      [-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1], [0, 0, 0]], dtype=np.int64)
PRISM18_REF = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1], [1, -1, 1], [-1, 1, 1],
                        [0, -1, -1], [0, 0, -1], [-1, 0, -1], [0, -1, 1], [0, 0, 1], [-1, 0, 1],
                        [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [0, -1, 0], [0, 0, 0], [-1, 0, 0]], dtype=np.int64)


def _tri_bary(r, s):
    return np.array([-(r + s) / 2.0, (1.0 + r) / 2.0, (1.0 + s) / 2.0])


def hex27_rotation_permutations() -> np.ndarray:
    """[24][27]: the node relabelling of each cube rotation (new node k = old node perm[r][k])."""
    lookup = {tuple(v): i for i, v in enumerate(HEX27_REF.tolist())}
    return np.array([[lookup[tuple((R @ c).tolist())] for c in HEX27_REF] for R in cube_rotations()], dtype=np.int64)


def prism18_permutations() -> np.ndarray:
    """[6][18]: node relabelling of each PRISM_PERMUTATIONS entry (new node k = old node perm[q][k])."""
    lookup = {}
    for i, (r, s, z) in enumerate(PRISM18_REF.tolist()):
        lookup[tuple(np.round(_tri_bary(r, s), 6).tolist()) + (z,)] = i
    out = []
    for P in PRISM_PERMUTATIONS:
        flip = P[0] >= 3
        row = []
        for (r, s, z) in PRISM18_REF.tolist():
            lam_new = _tri_bary(r, s)
            lam_old = np.zeros(3)
            for k in range(3):
                lam_old[P[k] % 3] = lam_new[k]
            row.append(lookup[tuple(np.round(lam_old, 6).tolist()) + ((-z if flip else z),)])
        out.append(row)
    return np.array(out, dtype=np.int64)


def curved_box_mesh(n: Sequence[int], lo=(0.0, 0.0, 0.0), hi=(2 * np.pi,) * 3, periodic=(True, True, True),
                    warp: float = 0.1, seed: int | None = None, shuffle: bool = False, rotate: bool = False,
                    wall_tags: dict | None = None, prisms=None) -> MeshDesc:
    """Box of nx*ny*nz quadratic (27-node) hexahedra, or 18-node prisms where columns are split like
    `hex_box_mesh`, on a (2n+1)^3 node lattice whose every node x is moved by the smooth periodic
    warp d_a(x) = warp L_a / (2 pi) sin(2 pi (x_b - lo_b) / L_b) sin(2 pi (x_c - lo_c) / L_c) ((a, b, c)
    cyclic), so element faces are curved (also on non-periodic boundaries).  Tags, periodic pairs,
    `rotate` (the 24 cube rotations / 6 prism relabellings applied to all nodes), `shuffle` and
    `wall_tags` as in `hex_box_mesh`; boundary faces list their corner nodes."""
    nx, ny, nz = (int(v) for v in n)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    L = hi - lo
    rng = np.random.default_rng(seed if seed is not None else 0)
    xs = [np.linspace(lo[a], hi[a], 2 * m + 1) for a, m in enumerate((nx, ny, nz))]
    X, Y, Z = np.meshgrid(xs[0], xs[1], xs[2], indexing="ij")
    P = np.stack([X, Y, Z], axis=-1).reshape(-1, 3)
    th = 2 * np.pi * (P - lo[None, :]) / L[None, :]
    d = np.empty_like(P)
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        d[:, a] = warp * L[a] / (2 * np.pi) * np.sin(th[:, b]) * np.sin(th[:, c])
    xyz = P + d
    nid = np.arange(xyz.shape[0]).reshape(2 * nx + 1, 2 * ny + 1, 2 * nz + 1)
    split = np.zeros((nx, ny), dtype=bool)
    if prisms == "all":
        split[:] = True
    elif prisms == "checker":
        split[(np.add.outer(np.arange(nx), np.arange(ny)) % 2) == 0] = True
    hexes, pris = [], []
    # prism A covers hex corners (-1,-1), (1,-1), (1,1) of the bottom face, prism B (-1,-1), (1,1), (-1,1)
    tri_corners = (np.array([[-1, -1], [1, -1], [1, 1]]), np.array([[-1, -1], [1, 1], [-1, 1]]))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                base = np.array([2 * i + 1, 2 * j + 1, 2 * k + 1])
                if not split[i, j]:
                    hexes.append([nid[tuple(base + c)] for c in HEX27_REF])
                    continue
                for V in tri_corners:
                    row = []
                    for (r, s, z) in PRISM18_REF.tolist():
                        lam = _tri_bary(r, s)
                        pxy = (lam[:, None] * V).sum(axis=0)
                        row.append(nid[base[0] + int(round(pxy[0])), base[1] + int(round(pxy[1])), base[2] + z])
                    pris.append(row)
    hexes = np.array(hexes, dtype=np.int64).reshape(-1, 27)
    pris = np.array(pris, dtype=np.int64).reshape(-1, 18)
    # Boundary faces (corner nodes), tags 1..6.
    bnodes, btags = [], []
    c = lambda I, J, K: nid[2 * I, 2 * J, 2 * K]   # noqa: E731  corner lattice node
    for j in range(ny):
        for k in range(nz):
            bnodes.append([c(0, j, k), c(0, j + 1, k), c(0, j + 1, k + 1), c(0, j, k + 1)]); btags.append(1)
            bnodes.append([c(nx, j, k), c(nx, j + 1, k), c(nx, j + 1, k + 1), c(nx, j, k + 1)]); btags.append(2)
    for i in range(nx):
        for k in range(nz):
            bnodes.append([c(i, 0, k), c(i + 1, 0, k), c(i + 1, 0, k + 1), c(i, 0, k + 1)]); btags.append(3)
            bnodes.append([c(i, ny, k), c(i + 1, ny, k), c(i + 1, ny, k + 1), c(i, ny, k + 1)]); btags.append(4)
    for i in range(nx):
        for j in range(ny):
            for kk, tag in ((0, 5), (nz, 6)):
                q = [c(i, j, kk), c(i + 1, j, kk), c(i + 1, j + 1, kk), c(i, j + 1, kk)]
                if split[i, j]:
                    bnodes.append([q[0], q[1], q[2], -1]); btags.append(tag)
                    bnodes.append([q[0], q[2], q[3], -1]); btags.append(tag)
                else:
                    bnodes.append(q); btags.append(tag)
    per = []
    for a in range(3):
        if periodic[a]:
            t = np.zeros(3)
            t[a] = float(L[a])
            per.append(Periodic(2 * a + 1, 2 * a + 2, tuple(float(v) for v in t)))
    bcs = []
    if wall_tags:
        for tag, (kind, params) in wall_tags.items():
            bcs.append(BC(int(tag), int(kind), tuple(float(v) for v in params)))
    if rotate:
        if len(hexes):
            r = rng.integers(0, 24, size=hexes.shape[0])
            hexes = np.take_along_axis(hexes, hex27_rotation_permutations()[r], axis=1)
        if len(pris):
            r = rng.integers(0, 6, size=pris.shape[0])
            pris = np.take_along_axis(pris, prism18_permutations()[r], axis=1)
    if shuffle:
        hexes = hexes[rng.permutation(hexes.shape[0])]
        pris = pris[rng.permutation(pris.shape[0])]
    return MeshDesc(xyz=np.ascontiguousarray(xyz, dtype=np.float64), hex=np.ascontiguousarray(hexes),
                    bface_nodes=np.array(bnodes, dtype=np.int64).reshape(-1, 4),
                    bface_tag=np.array(btags, dtype=np.int32), periodic=per, bcs=bcs,
                    prism=np.ascontiguousarray(pris))


# Boundary tags of the blade passage.
TAG_INLET, TAG_OUTLET, TAG_PER_LO, TAG_PER_HI, TAG_SPAN_LO, TAG_SPAN_HI, TAG_SUCTION, TAG_PRESSURE = 1, 2, 3, 4, 5, 6, 7, 8


def blade_profile(seed: int = 0, thickness: float = 0.12):
    """NACA-4-digit-like section of unit chord with camber drawn from the seed: (camber line y_c,
    its slope, half thickness t) as functions of x in [0, 1] (closed trailing edge)."""
    rng = np.random.default_rng(seed)
    m = rng.uniform(0.03, 0.05)            # maximum camber
    pc = rng.uniform(0.35, 0.45)           # its chordwise position

    def yc(x):
        x = np.asarray(x, dtype=np.float64)
        return np.where(x < pc, m / pc ** 2 * (2 * pc * x - x * x), m / (1 - pc) ** 2 * ((1 - 2 * pc) + 2 * pc * x - x * x))

    def t(x):
        x = np.clip(np.asarray(x, dtype=np.float64), 0.0, 1.0)
        return 5 * thickness * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2 + 0.2843 * x ** 3 - 0.1036 * x ** 4)
    return yc, t, m, pc


def blade_passage_mesh(n_up: int = 25, n_blade: int = 75, n_down: int = 25, ny: int = 70, nz: int = 40,
                       n_prism_rows: int = 8, pitch: float = 0.8, span: float = 0.3, stagger_deg: float = 30.0,
                       x_in: float = -0.6, x_out: float = 1.6, seed: int = 0, quadratic: bool = True,
                       bcs=None) -> MeshDesc:
    """Synthetic linear-cascade passage (unit chord): an H-mesh between the suction side of one
    blade and the pressure side of the next (a pitch above), sheared by the stagger angle
    (y -> y + x tan(stagger)), extruded over `span` in z with nz layers.  Upstream and downstream
    of the blade the lower and upper boundaries are periodic (translation (0, pitch, 0)); z is
    periodic (translation (0, 0, span)).  Cells within n_prism_rows of either blade surface (over
    the chord) are split into two prisms each.  With quadratic elements every node of the
    (2 nx + 1) x (2 ny + 1) x (2 nz + 1) lattice lies on the analytic map, so wall faces follow the
    blade surface to second order.  Tags: TAG_INLET / TAG_OUTLET, TAG_PER_LO / TAG_PER_HI,
    TAG_SPAN_LO / TAG_SPAN_HI, TAG_SUCTION / TAG_PRESSURE (walls); `bcs` maps tags to
    (kind, params) for the non-periodic ones."""
    yc, t, _, _ = blade_profile(seed)
    nx = n_up + n_blade + n_down
    q = 2 if quadratic else 1
    # Streamwise lattice coordinate: uniform upstream/downstream, mildly clustered at the leading
    # and trailing edges on the blade (30 % cosine, 70 % uniform: aspect ratios stay below ~2, so
    # the volume-based element size is close to the shortest edge).
    u_up = np.linspace(x_in, 0.0, q * n_up + 1)
    ub = np.linspace(0.0, 1.0, q * n_blade + 1)
    u_bl = 0.3 * 0.5 * (1 - np.cos(np.pi * ub)) + 0.7 * ub
    u_dn = np.linspace(1.0, x_out, q * n_down + 1)
    X1 = np.concatenate([u_up, u_bl[1:], u_dn[1:]])                       # [q nx + 1]
    on_blade = (X1 >= 0.0) & (X1 <= 1.0)
    y_lo = np.where(on_blade, yc(np.clip(X1, 0, 1)) + t(X1), 0.0)
    y_hi = np.where(on_blade, yc(np.clip(X1, 0, 1)) - t(X1), 0.0) + pitch
    eta = np.linspace(0.0, 1.0, q * ny + 1)
    eta = 0.5 * (1 - np.cos(np.pi * eta)) * 0.5 + 0.5 * eta               # mild clustering at both walls
    zz = np.linspace(0.0, span, q * nz + 1)
    XX = np.broadcast_to(X1[:, None, None], (X1.size, eta.size, zz.size))
    YY = y_lo[:, None, None] + eta[None, :, None] * (y_hi - y_lo)[:, None, None]
    ZZ = np.broadcast_to(zz[None, None, :], XX.shape)
    YY = YY + np.tan(np.radians(stagger_deg)) * XX
    xyz = np.stack([A.transpose(2, 1, 0).ravel() for A in (XX, YY, ZZ)], 1)   # node I + NI (J + NJ K)
    NI, NJ = q * nx + 1, q * ny + 1
    nid = lambda I, J, K: I + NI * (J + NJ * K)   # noqa: E731
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    blade_col = (ci >= n_up) & (ci < n_up + n_blade)
    split = blade_col & ((cj < n_prism_rows) | (cj >= ny - n_prism_rows))
    base = [q * ci + (1 if quadratic else 0), q * cj + (1 if quadratic else 0), q * ck + (1 if quadratic else 0)]
    if quadratic:
        href, pref = HEX27_REF, PRISM18_REF
        off = lambda c: c                   # noqa: E731  reference coordinate -> lattice offset
    else:
        href, pref = HEX_REF_VERTS.astype(np.int64), PRISM18_REF[:6]
        off = lambda c: (c + 1) // 2        # noqa: E731
    hsel = ~split
    hexes = np.stack([nid(base[0][hsel] + off(c[0]), base[1][hsel] + off(c[1]), base[2][hsel] + off(c[2]))
                      for c in href], 1)
    pris = []
    for V in (np.array([[-1, -1], [1, -1], [1, 1]]), np.array([[-1, -1], [1, 1], [-1, 1]])):
        cols = []
        for (r, s_, z) in pref.tolist():
            lam = _tri_bary(r, s_)
            pxy = np.round((lam[:, None] * V).sum(axis=0)).astype(np.int64)
            cols.append(nid(base[0][split] + off(pxy[0]), base[1][split] + off(pxy[1]), base[2][split] + off(z)))
        pris.append(np.stack(cols, 1))
    pris = np.stack(pris, 1).reshape(-1, pref.shape[0])                   # the two prisms of a cell adjacent
    # Boundary faces (corner nodes).
    c = lambda I, J, K: nid(q * I, q * J, q * K)   # noqa: E731
    bn, bt = [], []
    J, K = np.meshgrid(np.arange(ny), np.arange(nz), indexing="ij")
    J, K = J.ravel(), K.ravel()
    for I0, tag in ((0, TAG_INLET), (nx, TAG_OUTLET)):
        bn.append(np.stack([c(I0, J, K), c(I0, J + 1, K), c(I0, J + 1, K + 1), c(I0, J, K + 1)], 1)); bt.append(np.full(J.size, tag))
    Iw, K = np.meshgrid(np.arange(nx), np.arange(nz), indexing="ij")
    Iw, K = Iw.ravel(), K.ravel()
    wall = (Iw >= n_up) & (Iw < n_up + n_blade)
    for J0, tw, tp in ((0, TAG_SUCTION, TAG_PER_LO), (ny, TAG_PRESSURE, TAG_PER_HI)):
        bn.append(np.stack([c(Iw, J0, K), c(Iw + 1, J0, K), c(Iw + 1, J0, K + 1), c(Iw, J0, K + 1)], 1))
        bt.append(np.where(wall, tw, tp))
    Ic, Jc = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    Ic, Jc = Ic.ravel(), Jc.ravel()
    sp = ((Ic >= n_up) & (Ic < n_up + n_blade)) & ((Jc < n_prism_rows) | (Jc >= ny - n_prism_rows))
    for K0, tag in ((0, TAG_SPAN_LO), (nz, TAG_SPAN_HI)):
        qd = np.stack([c(Ic, Jc, K0), c(Ic + 1, Jc, K0), c(Ic + 1, Jc + 1, K0), c(Ic, Jc + 1, K0)], 1)
        bn.append(qd[~sp]); bt.append(np.full((~sp).sum(), tag))
        m1 = -np.ones(sp.sum(), dtype=np.int64)
        bn.append(np.stack([qd[sp, 0], qd[sp, 1], qd[sp, 2], m1], 1)); bt.append(np.full(sp.sum(), tag))
        bn.append(np.stack([qd[sp, 0], qd[sp, 2], qd[sp, 3], m1], 1)); bt.append(np.full(sp.sum(), tag))
    per = [Periodic(TAG_PER_LO, TAG_PER_HI, (0.0, float(pitch), 0.0)), Periodic(TAG_SPAN_LO, TAG_SPAN_HI, (0.0, 0.0, float(span)))]
    bc_list = [BC(int(tag), int(kind), tuple(float(v) for v in params)) for tag, (kind, params) in (bcs or {}).items()]
    return MeshDesc(xyz=np.ascontiguousarray(xyz), hex=np.ascontiguousarray(hexes.astype(np.int64)),
                    bface_nodes=np.ascontiguousarray(np.concatenate(bn).astype(np.int64)),
                    bface_tag=np.concatenate(bt).astype(np.int32), periodic=per, bcs=bc_list,
                    prism=np.ascontiguousarray(pris.astype(np.int64)))


def cascade_conditions(Ma_in: float = 0.15, Ma_exit: float = 0.9, Re: float = 5e5, gamma: float = 1.4,
                       stagger_deg: float = 30.0):
    """Physics and boundary data of the synthetic cascade (unit chord, p0 = rho0 = 1, R = 1, so
    T0 = 1): characteristic inflow with total conditions along the stagger direction, static
    back-pressure from the isentropic exit Mach number, isothermal blade walls at T0, mu from the
    Reynolds number on chord and isentropic exit speed.  Returns (Physics, bcs, inflow state fn)."""
    R = 1.0
    T0 = p0 = 1.0
    f = lambda M: 1 + 0.5 * (gamma - 1) * M * M   # noqa: E731
    pb = p0 * f(Ma_exit) ** (-gamma / (gamma - 1))
    Te = T0 / f(Ma_exit)
    Ue = Ma_exit * np.sqrt(gamma * R * Te)
    rho_e = pb / (R * Te)
    mu = rho_e * Ue * 1.0 / Re
    d = (np.cos(np.radians(stagger_deg)), np.sin(np.radians(stagger_deg)), 0.0)
    phys = Physics(gamma=gamma, R=R, mu=mu, Pr=0.71, viscous=1)
    bcs = {TAG_INLET: (BC_CHAR_INFLOW, (p0, T0) + d), TAG_OUTLET: (BC_CHAR_OUTFLOW, (pb,)),
           TAG_SUCTION: (BC_WALL_ISOTHERMAL, (T0,)), TAG_PRESSURE: (BC_WALL_ISOTHERMAL, (T0,))}
    Ti = T0 / f(Ma_in)
    pi = p0 * f(Ma_in) ** (-gamma / (gamma - 1))
    Ui = Ma_in * np.sqrt(gamma * R * Ti)

    def state(x, perturb=1e-3, seed=0):
        """Uniform inflow state with a seeded random-phase velocity perturbation."""
        rng = np.random.default_rng(seed)
        ph_ = rng.uniform(0, 2 * np.pi, 3)
        k = 2 * np.pi * np.array([1.0, 1 / 0.8, 1 / 0.3])
        dv = perturb * Ui * np.stack([np.sin(k[0] * x[..., 0] + ph_[0]) * np.cos(k[1] * x[..., 1]),
                                      np.sin(k[1] * x[..., 1] + ph_[1]) * np.cos(k[2] * x[..., 2]),
                                      np.sin(k[2] * x[..., 2] + ph_[2]) * np.cos(k[0] * x[..., 0])], -1)
        u = Ui * np.asarray(d)[None] * np.ones(x.shape[:-1] + (1,)) + dv
        rho = pi / (R * Ti) * np.ones(x.shape[:-1])
        return conserved(rho, u[..., 0], u[..., 1], u[..., 2], pi * np.ones(x.shape[:-1]), gamma)
    return phys, bcs, state


# ---------------------------------------------------------------------------------------------
# Physical parameters and initial conditions (functions of physical coordinates only).
# ---------------------------------------------------------------------------------------------

@dataclass
class Physics:
    gamma: float = 1.4
    R: float = 1.0
    mu: float = 0.0
    Pr: float = 0.71
    inviscid_flux: int = 0      # 0 = Rusanov, 1 = Roe
    viscous: int = 1            # 0 = Euler, 1 = BR2, 2 = LDG
    br2_eta: float = 6.0
    ldg_tau: float = 0.1        # LDG penalty
    vcjh_c: float = 0.0
    precision: int = 0          # 0 = FP64, 1 = double-float element operators, 2 = the same with the face
                                # interpolation on the tensor cores, 3 = with the viscous branch in FP32


def tgv_physics(Ma: float = 0.1, Re: float = 1600.0, gamma: float = 1.4, Pr: float = 0.71) -> Physics:
    """Taylor-Green vortex in units rho0 = V0 = L = T0 = 1, p0 = 1/(gamma Ma^2), R = p0."""
    p0 = 1.0 / (gamma * Ma * Ma)
    return Physics(gamma=gamma, R=p0, mu=1.0 / Re, Pr=Pr, viscous=1, br2_eta=6.0)


def conserved(rho, u, v, w, p, gamma):
    """Stack primitive fields into conserved variables (rho, rho u, rho v, rho w, E) on the last axis."""
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)
    return np.stack([rho, rho * u, rho * v, rho * w, E], axis=-1)


def tgv_state(x: np.ndarray, Ma: float = 0.1, gamma: float = 1.4, perturb: float = 0.0,
              seed: int = 0) -> np.ndarray:
    """Taylor-Green vortex at points x[..., 3] (conserved variables on the last axis).

    Velocity u = sin x cos y cos z, v = -cos x sin y cos z, w = 0; pressure
    p = p0 + (cos 2x + cos 2y)(cos 2z + 2)/16 with p0 = 1/(gamma Ma^2); density from the ideal
    gas law at uniform temperature T0 = 1 (R = p0).  `perturb` > 0 adds a seeded sum of
    random-phase Fourier modes (wavenumbers 1..3) of that amplitude to the three velocities.
    """
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    p0 = 1.0 / (gamma * Ma * Ma)
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(X)
    p = p0 + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    if perturb > 0.0:
        rng = np.random.default_rng(seed)
        vel = [u, v, w]
        for c in range(3):
            for _ in range(4):
                kv = rng.integers(1, 4, size=3)
                ph = rng.uniform(0, 2 * np.pi)
                vel[c] = vel[c] + perturb * np.sin(kv[0] * X + kv[1] * Y + kv[2] * Z + ph)
        u, v, w = vel
    rho = p / p0
    return conserved(rho, u, v, w, p, gamma)


def isentropic_vortex_state(x: np.ndarray, t: float = 0.0, centre=(0.0, 0.0), beta: float = 5.0,
                            Ma: float = 0.5, direction=(1.0, 1.0), gamma: float = 1.4,
                            period=None) -> np.ndarray:
    """Isentropic (Shu-type) vortex in the x-y plane, uniform in z, exact for the Euler equations.

    Free stream rho = 1, p = 1 (so T = p/rho = 1 with R = 1) and speed Ma * sqrt(gamma) along
    `direction`.  The perturbation about the advected centre is
    du = -beta/(2 pi) e^{(1-r^2)/2} (y - yc), dv = beta/(2 pi) e^{(1-r^2)/2} (x - xc),
    dT = -(gamma-1) beta^2/(8 gamma pi^2) e^{1-r^2}, with rho = T^{1/(gamma-1)}, p = rho T.
    With `period` = (Lx, Ly) the nearest periodic image of the centre is used.
    """
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    U = Ma * np.sqrt(gamma)
    u0, v0 = U * d[0], U * d[1]
    xc = centre[0] + u0 * t
    yc = centre[1] + v0 * t
    dx = x[..., 0] - xc
    dy = x[..., 1] - yc
    if period is not None:
        dx = dx - period[0] * np.round(dx / period[0])
        dy = dy - period[1] * np.round(dy / period[1])
    r2 = dx * dx + dy * dy
    f = np.exp(0.5 * (1.0 - r2))
    u = u0 - beta / (2 * np.pi) * f * dy
    v = v0 + beta / (2 * np.pi) * f * dx
    T = 1.0 - (gamma - 1.0) * beta * beta / (8.0 * gamma * np.pi * np.pi) * f * f
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho * T
    return conserved(rho, u, v, np.zeros_like(u), p, gamma)


def uniform_state(shape, rho=1.0, vel=(0.3, 0.2, 0.1), p=None, gamma=1.4) -> np.ndarray:
    """Uniform flow (free stream) of the given shape; default p = 1/gamma."""
    if p is None:
        p = 1.0 / gamma
    one = np.ones(shape)
    return conserved(rho * one, vel[0] * one, vel[1] * one, vel[2] * one, p * one, gamma)


def vortex_ensemble(n_cases: int = 64, seed0: int = 0):
    """Case list of a batched isentropic-vortex ensemble: per case i (seed i) an edge count
    n ~ U{8..24}, an order p ~ U{2..5} and a vortex centre ~ U(domain), all from splitmix64."""
    cases = []
    for i in range(n_cases):
        r = splitmix64_uniform(seed0 + i, 4)
        n = 8 + int(r[0] * 17)
        p = 2 + int(r[1] * 4)
        L = 20.0
        cases.append(dict(seed=seed0 + i, n=n, p=p, L=L,
                          centre=(-L / 2 + L * r[2], -L / 2 + L * r[3])))
    return cases
