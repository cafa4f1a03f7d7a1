"""Host analysis: Fourier transform of class sums, rebinning and jackknife."""
import numpy as np
import pytest

from paper_1704_00131_gb300 import analysis as A
from paper_1704_00131_gb300 import workloads as W


def test_fourier_of_class_sums_matches_direct_double_sum():
    Lx, Ly = 4, 3
    N = Lx * Ly
    rng = np.random.default_rng(0)
    M = rng.standard_normal((N, N))                 # any pair function
    cls, n, r = W.translation_classes_square(Lx, Ly)
    C = np.bincount(cls, weights=M.ravel(), minlength=n)
    q = A.momenta_square(Lx, Ly)
    S = A.fourier(C, r, q, N)
    pos = np.array([[i % Lx, i // Lx] for i in range(N)], dtype=float)
    for k, qk in enumerate(q):
        direct = sum(np.exp(1j * qk @ (pos[j] - pos[i])) * M[i, j] for i in range(N) for j in range(N)) / N
        assert S[k] == pytest.approx(direct, abs=1e-12)


def test_jackknife_unit_sign_is_the_standard_error():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(400) + 3.0
    bins = A.rebin(x, 20)
    mean, err = A.jackknife(bins, np.ones(20))
    assert mean == pytest.approx(bins.mean(), abs=1e-14)
    assert err == pytest.approx(bins.std(ddof=1) / np.sqrt(20), rel=1e-12)


def test_jackknife_sign_reweighting():
    rng = np.random.default_rng(2)
    s = np.where(rng.random(4000) < 0.8, 1.0, -1.0)
    o = rng.standard_normal(4000) + 1.0
    ob, sb = A.rebin(o * s, 40), A.rebin(s, 40)
    mean, err = A.jackknife(ob[:, None], sb)
    assert mean[0] == pytest.approx((o * s).sum() / s.sum(), rel=1e-12)
    assert 0 < err[0] < 1.0
    with pytest.raises(ValueError):
        A.rebin(o, 5000)
    with pytest.raises(ValueError):
        A.jackknife(ob[:1], sb[:1])
