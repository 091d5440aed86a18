"""The synthetic cascade passage at full size (398 000 quadratic elements, 24 % prisms, p = 7,
182 M solution points) on the GPU, checked on sampled elements against the oracle (marked gpu).

BR2 is compact: an element's residual depends only on its own state and its face neighbours'.
Each sample is evaluated by the oracle on a patch made of the element and its face neighbours;
the patch's outer faces get a Dirichlet condition (any state: it cannot reach the sample), the
real walls and in/outflow faces keep their conditions.  The state is a function of the element
and point indices, so the patch's state is the full mesh's restricted.  Samples avoid the
periodic boundaries (middle span layers, prisms at the walls, hexahedra inside the passage and at
the inlet and outlet).
"""
import numpy as np
import pytest

from paper_2308_06605_gb300 import fr
from paper_2308_06605_gb300 import inputs as I
from oracle.mixedfr import MixedFR, hex_type, prism_type

from helpers import assert_residual_parity, ensure_lib

pytestmark = pytest.mark.gpu

P = 7
NZ = 40
PERIODIC_TAGS = (I.TAG_PER_LO, I.TAG_PER_HI, I.TAG_SPAN_LO, I.TAG_SPAN_HI)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def _state(base, elem, npts, offset):
    """Base state times a smooth pattern in the (element, point) indices: [len(elem)][npts][5]."""
    e = np.asarray(elem, dtype=np.float64)[:, None]
    m = np.arange(npts, dtype=np.float64)[None, :]
    Q = np.empty((len(elem), npts, 5))
    for v in range(5):
        Q[..., v] = base[v] * (1 + 2e-3 * np.sin(0.37 * e + 1.31 * m + 0.7 * v + offset))
    return Q


def _patch(d, sample, is_prism, bkeys):
    """The sample element and its face neighbours: (mesh, global hex ids, global prism ids)."""
    own = (d.prism if is_prism else d.hex)[sample]
    faces = prism_type(1).faces if is_prism else hex_type(1).faces
    hx_ids, pr_ids = ([], [sample]) if is_prism else ([sample], [])
    for f in faces:
        key = own[f["corners"]]
        for arr, ids, ncorner in ((d.hex, hx_ids, 8), (d.prism, pr_ids, 6)):
            hit = np.where(np.isin(arr[:, :ncorner], key).sum(axis=1) == len(key))[0]
            ids += [int(h) for h in hit if int(h) not in ids]
    hexes, pris = d.hex[hx_ids], d.prism[pr_ids]
    nodes = np.unique(np.concatenate([hexes.ravel(), pris.ravel()]))
    remap = np.full(d.xyz.shape[0], -1, dtype=np.int64)
    remap[nodes] = np.arange(nodes.size)
    hx, pp = remap[hexes].reshape(-1, 27), remap[pris].reshape(-1, 18)
    count = {}
    for arr, ft in ((hx, hex_type(1).faces), (pp, prism_type(1).faces)):
        for row in arr:
            for f in ft:
                k = tuple(sorted(row[f["corners"]].tolist()))
                count[k] = count.get(k, 0) + 1
    bn, bt = [], []
    for k, c in count.items():
        if c == 2:
            continue
        tag = bkeys.get(tuple(sorted(int(nodes[i]) for i in k)), 99)
        bn.append(list(k) + ([-1] if len(k) == 3 else []))
        bt.append(tag)
    bcs = [b for b in d.bcs if b.tag in set(bt)] + [I.BC(99, I.BC_DIRICHLET, (1.0, 0.1, 0.0, 0.0, 2.5))]
    desc = I.MeshDesc(xyz=d.xyz[nodes], hex=hx, bface_nodes=np.array(bn, dtype=np.int64).reshape(-1, 4),
                      bface_tag=np.array(bt, dtype=np.int32), periodic=[], bcs=bcs, prism=pp)
    return desc, hx_ids, pr_ids


@pytest.mark.parametrize("precision,rel", [(0, 1e-12), (1, 1e-9)])
def test_cascade_p7_full_size_sampled(precision, rel):
    phys, bcs, state_fn = I.cascade_conditions()
    phys.precision = precision
    d = I.blade_passage_mesh(nz=NZ, bcs=bcs)
    E, Ep = len(d.hex), len(d.prism)
    Nh, Npr = (P + 1) ** 3, (P + 1) * (P + 1) * (P + 2) // 2
    base = state_fn(np.zeros((1, 3)), perturb=0.0)[0]
    Q = np.ascontiguousarray(np.concatenate([_state(base, np.arange(E), Nh, 0.0).reshape(-1, 5),
                                             _state(base, np.arange(Ep), Npr, 1.0).reshape(-1, 5)]))
    with fr.Mesh(d, phys, P) as g:
        assert g.n_elem == E and g.n_prism == Ep and g.n_points == E * Nh + Ep * Npr == 182_272_000
        g.set_state(Q)
        R = g.residual()
    del Q
    assert np.isfinite(R).all()
    Rh, Rp = R[:E * Nh].reshape(E, Nh, 5), R[E * Nh:].reshape(Ep, Npr, 5)
    bkeys = {tuple(sorted(int(v) for v in row if v >= 0)): int(t) for row, t in zip(d.bface_nodes, d.bface_tag)}
    # Samples by corner centroid: middle span, hexahedra inside the passage and in the first and
    # last columns (inflow, outflow), prisms (they line the blade walls).
    ch, cp = d.xyz[d.hex[:, :8]].mean(axis=1), d.xyz[d.prism[:, :6]].mean(axis=1)
    span = ch[:, 2].max() + ch[:, 2].min()
    mid_h = np.abs(ch[:, 2] - span / 2) < 0.3 * span
    mid_p = np.abs(cp[:, 2] - span / 2) < 0.3 * span
    rng = np.random.default_rng(0)
    pick = lambda mask, k: [int(v) for v in rng.choice(np.where(mask)[0], size=k, replace=False)]  # noqa: E731
    samples = ([(False, e) for e in pick(mid_h & (ch[:, 0] > 0.2) & (ch[:, 0] < 0.8), 4)] +
               [(False, e) for e in pick(mid_h & (ch[:, 0] < ch[:, 0].min() + 1e-3), 3)] +
               [(False, e) for e in pick(mid_h & (ch[:, 0] > ch[:, 0].max() - 1e-3), 3)] +
               [(True, e) for e in pick(mid_p, 6)])
    checked = 0
    ph_ora = I.Physics(**{f: getattr(phys, f) for f in phys.__dataclass_fields__})
    ph_ora.precision = 0
    for is_prism, s in samples:
        desc, hx_ids, pr_ids = _patch(d, s, is_prism, bkeys)
        if any(int(t) in PERIODIC_TAGS for t in desc.bface_tag):
            continue
        ora = MixedFR(desc, ph_ora, P)
        Qs = [_state(base, hx_ids, Nh, 0.0), _state(base, pr_ids, Npr, 1.0)]
        Ro = ora.residual(Qs)
        So = ora.residual(Qs, magnitude=True)
        t = 1 if is_prism else 0
        assert_residual_parity((Rp if is_prism else Rh)[s], Ro[t][0], So[t][0], rel=rel)
        checked += 1
    assert checked >= 8
