"""Pins of the SVD-stabilised UDV chain (orc_green_udv_svd, the stabilisation
option by singular value decomposition): G, log|det| and sign equal those of
the column-pivoted QR chain at beta = 10 and U = 6, and the plain product at
beta = 2 for an interior tau.  Two backward-stable routes to the same inverse
agree to rounding times its conditioning, which grows with the size of G's
entries (up to ~10 with the four-valued field at U = 6), so the comparison is
relative to max(1, max|G|)."""
import numpy as np
import pytest

from paper_1704_00131_gb300 import workloads as W


def omodel(orc, m):
    return orc.Model(m.hopping, m.vertex_site, m.vertex_sign, m.U, m.dtau, m.L, m.n_wrap, m.field_type)


@pytest.mark.parametrize("ft", [1, 2])
def test_svd_chain_equals_qr_chain_at_large_beta(orc, ft):
    m = W.ModelSpec(W.square_lattice(4, 4, tp=-0.1, mu=-0.2), U=6.0, dtau=0.1, L=100, n_wrap=10, field_type=ft)
    om = omodel(orc, m)
    f = W.random_fields(ft, m.L, 16, seed=3)
    for s in (0, 1):
        for tau in (0, 37):
            Gq, lq, sq = orc.green_udv(om, f, s, tau)
            Gs, ls, ss = orc.green_udv_svd(om, f, s, tau)
            assert np.abs(Gq - Gs).max() < 1e-10 * max(1.0, np.abs(Gq).max()), (s, tau)
            assert ls == pytest.approx(lq, rel=1e-12) and ss == sq


def test_svd_chain_equals_plain_product(orc):
    m = W.ModelSpec(W.honeycomb_lattice(2, 2), U=4.0, dtau=0.1, L=20, n_wrap=5)
    om = omodel(orc, m)
    f = W.random_fields(1, m.L, m.N, seed=4)
    for s in (0, 1):
        Gp, lp, sp = orc.green_plain(om, f, s, 7)
        Gs, ls, ss = orc.green_udv_svd(om, f, s, 7)
        assert np.abs(Gp - Gs).max() < 5e-11
        assert ls == pytest.approx(lp, rel=1e-10) and ss == sp
