"""The library's host-computed 1D tables (fr_basis_1d: Golub-Welsch nodes, barycentric
derivative matrix, correction vectors as the DG lifting l_i(+-1)/w_i plus the energy-stable
family's -kappa P_p term) against the oracle's independent construction (Newton nodes,
product-formula Lagrange derivatives, g_R' of the family from the Legendre recurrences).  CPU
only: the call does no device work."""
import numpy as np
import pytest

from oracle.basis import Basis1D
from paper_2308_06605_gb300 import build as B
from paper_2308_06605_gb300 import fr

from helpers import vcjh_c


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(fr.LIB_PATH):
        B.build()
    fr.load()


@pytest.mark.parametrize("which", ["dg", "sd", "hu", "neg", "big"])
@pytest.mark.parametrize("p", range(1, 8))
def test_library_tables_match_oracle(p, which):
    c = vcjh_c(p, which)
    lib = fr.basis_1d(p, c)
    ora = Basis1D(p, c)
    np.testing.assert_allclose(lib["x"], ora.nodes, rtol=0, atol=1e-15)
    np.testing.assert_allclose(lib["w"], ora.weights, rtol=1e-14, atol=0)
    scale = np.abs(ora.D).max()
    np.testing.assert_allclose(lib["D"], ora.D, rtol=0, atol=2e-14 * scale)
    np.testing.assert_allclose(lib["lm"], ora.l_minus, rtol=0, atol=1e-14)
    np.testing.assert_allclose(lib["lp"], ora.l_plus, rtol=0, atol=1e-14)
    hs = np.abs(ora.h_plus).max()
    np.testing.assert_allclose(lib["hp"], ora.h_plus, rtol=0, atol=1e-13 * hs)
    np.testing.assert_allclose(lib["hm"], ora.h_minus, rtol=0, atol=1e-13 * hs)


def test_out_of_range_refused():
    for p, c in ((0, 0.0), (8, 0.0), (3, 2.0 * vcjh_c(3, "neg") * 1.01), (2, float("nan"))):
        with pytest.raises(fr.FRError):
            fr.basis_1d(p, c)


@pytest.mark.parametrize("p", range(1, 8))
def test_library_triangle_tables_match_oracle(p):
    from oracle.tri import Tri
    lib = fr.tri_basis(p)
    T = Tri(p)
    np.testing.assert_allclose(lib["rs"], T.rs, rtol=0, atol=1e-14)
    sc = np.abs(T.Dr).max()
    np.testing.assert_allclose(lib["Dr"], T.Dr, rtol=0, atol=1e-13 * sc)
    np.testing.assert_allclose(lib["Ds"], T.Ds, rtol=0, atol=1e-13 * sc)
    Minv = np.linalg.inv(T.M)
    np.testing.assert_allclose(lib["Minv"], Minv, rtol=0, atol=1e-12 * np.abs(Minv).max())


@pytest.mark.parametrize("p,q", [(1, 3), (3, 1), (2, 2), (4, 7), (7, 4), (5, 6)])
def test_library_transfer_matrices_match_oracle(p, q):
    from oracle.project import line_transfer, tri_transfer
    np.testing.assert_allclose(fr.transfer_matrix(0, p, q), line_transfer(p, q), rtol=0, atol=1e-13)
    np.testing.assert_allclose(fr.transfer_matrix(1, p, q), tri_transfer(p, q), rtol=0, atol=1e-12)


def test_table_queries_refuse_bad_arguments():
    with pytest.raises(fr.FRError):
        fr.tri_basis(0)
    with pytest.raises(fr.FRError):
        fr.transfer_matrix(2, 2, 3)
    with pytest.raises(fr.FRError):
        fr.transfer_matrix(0, 2, 8)
