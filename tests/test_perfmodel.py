"""Algorithmic work model behind the roofline fractions (perfmodel.py), checked against counts
made independently here: the multiply-adds of the sum-factorised operators are counted by
walking one element's contractions, the bytes by listing the arrays each kernel reads and
writes once."""
import pytest

from paper_2308_06605_gb300 import perfmodel as PM


def _walk_macs(N, lines_per_point_dir, vars_, dirs):
    """Multiply-adds of applying a 1D operator of length N along `dirs` directions to `vars_`
    variables at every point of an N^3 element, counted point by point."""
    macs = 0
    for _pt in range(N ** 3):
        for _v in range(vars_):
            for _d in range(dirs):
                macs += N * lines_per_point_dir
    return macs


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_contraction_counts_match_a_walk_over_one_element(p):
    N = p + 1
    Np = N ** 3
    f = PM.flops_per_point(p, viscous=False)
    # inviscid volume: divergence (3 directions, 5 variables) + pointwise flux + transform
    div = 2 * _walk_macs(N, 1, 5, 3) / Np
    assert f["volume"] == pytest.approx(div + PM._INVISCID + PM._TRANSFORM)
    # face interpolation: 6 N^2 face points, 5 variables, N multiply-adds each
    interp = 2 * (6 * N * N) * 5 * N / Np
    assert f["interp_faces"] == pytest.approx(interp)
    # p = 4 figures quoted beside the measurements
    if p == 4:
        assert PM.flops_per_point(4)["volume"] == pytest.approx(987.0)
        assert f["interp_faces"] == pytest.approx(60.0)


@pytest.mark.parametrize("p", [1, 3, 4, 7])
def test_viscous_split_adds_up(p):
    visc, rest = PM.volume_split(p)
    assert visc + rest == pytest.approx(PM.flops_per_point(p)["volume"])
    assert rest == pytest.approx(PM.flops_per_point(p, viscous=False)["volume"])
    if p == 4:
        assert (round(visc), round(rest)) == (725, 262)


def test_mixed_peak_is_the_time_weighted_mix():
    df, f32 = 4.36, 78.5
    assert PM.mixed_alu_peak(4, df, f32, fp32_viscous=False) == df
    mix = PM.mixed_alu_peak(4, df, f32, fp32_viscous=True)
    assert df < mix < f32
    visc, rest = PM.volume_split(4)
    # time of the whole at the mixed peak equals the sum of the parts at their own peaks
    assert (visc + rest) / mix == pytest.approx(rest / df + visc / f32)


@pytest.mark.parametrize("p", [2, 4, 7])
def test_bytes_are_each_array_once(p):
    N = p + 1
    Np, Nf = N ** 3, N * N
    b = PM.bytes_per_point(p)
    per_el = 8.0 / Np
    # volume: state (5), metrics (9 S + 1/|J|), partial residual (5); both trace slots of the 6
    # faces (2 x 5 each), lift factors (3 per face point), gradient traces (15 per face point)
    vol = per_el * (5 * Np + 10 * Np + 5 * Np + 2 * 6 * Nf * 5 + 6 * 3 * Nf + 6 * 15 * Nf)
    assert b["volume"] == pytest.approx(vol)
    if p == 4:
        assert b["volume"] == pytest.approx(428.8)
    # interfaces (3 per element): two trace slots, normal (3 + |n|), common flux, two gradient slots
    assert b["iface_flux"] == pytest.approx(per_el * 3 * Nf * (10 + 4 + 5 + 30))
