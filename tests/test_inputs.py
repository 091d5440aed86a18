"""The seeded input generators shared by the oracle and the GPU path (CPU only): the counter-based
generator against the reference outputs of its published definition, reproducibility from seeds,
the ensemble's stated ranges, and the validity of the generated meshes (positive Jacobians at
every solution point, every boundary face tagged)."""
import numpy as np
import pytest

from paper_2308_06605_gb300 import inputs as I
from oracle.basis import Basis1D
from oracle.hexfr import trilinear_geometry


def test_splitmix64_reference_outputs():
    # First outputs of splitmix64 (Steele, Lea & Flood 2014; the reference implementation) from
    # state 0.
    got = [int(v) for v in I.splitmix64(0, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    u = I.splitmix64_uniform(7, 1000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.05


def test_vortex_ensemble_ranges_and_reproducibility():
    a, b = I.vortex_ensemble(64), I.vortex_ensemble(64)
    assert a == b
    assert all(8 <= c["n"] <= 24 and 2 <= c["p"] <= 5 for c in a)
    assert len({c["p"] for c in a}) == 4 and len({c["n"] for c in a}) > 8
    for c in a:
        assert all(-c["L"] / 2 <= x <= c["L"] / 2 for x in c["centre"])


@pytest.mark.parametrize("kw", [dict(seed=3, shuffle=True, rotate=True, perturb=0.15),
                                dict(seed=5, rotate=True, prisms="checker", perturb=0.1)])
def test_box_mesh_reproducible_and_valid(kw):
    d1, d2 = I.hex_box_mesh((4, 3, 2), **kw), I.hex_box_mesh((4, 3, 2), **kw)
    assert np.array_equal(d1.xyz, d2.xyz) and np.array_equal(d1.hex, d2.hex)
    if d1.prism is not None:
        assert np.array_equal(d1.prism, d2.prism)
    if len(d1.hex):
        xi = Basis1D(3).nodes
        K, J, Ii = np.meshgrid(xi, xi, xi, indexing="ij")
        ref = np.stack([Ii.ravel(), J.ravel(), K.ravel()], axis=1)
        _, detJ, _ = trilinear_geometry(d1.xyz[d1.hex], ref)
        assert np.all(detJ > 0)
    # every outer face is tagged and every tag is paired periodically (a fully periodic box)
    paired = {t for pp in d1.periodic for t in (pp.tag_a, pp.tag_b)}
    assert set(np.unique(d1.bface_tag)) <= paired and not d1.bcs


def test_walled_box_tags_every_boundary_face():
    d = I.hex_box_mesh((3, 2, 2), periodic=(False, True, True),
                       wall_tags={1: (I.BC_WALL_ISOTHERMAL, (1.0,)), 2: (I.BC_CHAR_OUTFLOW, (1.0,))})
    # outer faces: 2 x (2 x 2) at x = lo/hi, 2 x (3 x 2) in y and in z
    assert len(d.bface_tag) == 8 + 12 + 12
    assert np.sum(np.isin(d.bface_tag, [1, 2])) == 8
    paired = {t for pp in d.periodic for t in (pp.tag_a, pp.tag_b)}
    assert {b.tag for b in d.bcs} == {1, 2} and paired == {3, 4, 5, 6}
    assert set(np.unique(d.bface_tag)) == {1, 2} | paired
