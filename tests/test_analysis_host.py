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
    # Eq. jack_mean: the mean over i of the ratio without bin i
    loo = [(ob.sum() - ob[i]) / (sb.sum() - sb[i]) for i in range(40)]
    assert mean[0] == pytest.approx(np.mean(loo), rel=1e-12)
    assert err[0] == pytest.approx(np.sqrt(39 / 40 * np.sum((np.array(loo) - np.mean(loo)) ** 2)), rel=1e-12)
    assert mean[0] == pytest.approx((o * s).sum() / s.sum(), rel=1e-2)
    assert 0 < err[0] < 1.0
    with pytest.raises(ValueError):
        A.rebin(o, 5000)
    with pytest.raises(ValueError):
        A.jackknife(ob[:1], sb[:1])


A1, A2H = np.array([1.0, 0.0]), np.array([0.5, np.sqrt(3.0) / 2.0])     # triangular Bravais lattice


def test_reciprocal_vectors_and_momentum_grid():
    g1, g2 = A.reciprocal_vectors(A1, A2H)
    G = np.array([[A1 @ g1, A1 @ g2], [A2H @ g1, A2H @ g2]])
    assert np.abs(G - 2 * np.pi * np.eye(2)).max() < 1e-13
    # untilted square: the grid of momenta_square, in the same order
    assert np.abs(A.momenta([1, 0], [0, 1], [4, 0], [0, 3]) - A.momenta_square(4, 3)).max() < 1e-13
    # the honeycomb's triangular lattice, 6 x 6 cells, and a tilted sqrt(8) x sqrt(8) square lattice
    for a1, a2, L1, L2, n in ((A1, A2H, 6 * A1, 6 * A2H, 36),
                              (np.array([1.0, 0.0]), np.array([0.0, 1.0]), np.array([2.0, 2.0]), np.array([-2.0, 2.0]), 8)):
        k = A.momenta(a1, a2, L1, L2)
        assert k.shape == (n, 2)
        # allowed by the periodicity: e^{i k . L_i} = 1
        assert np.abs(np.exp(1j * (k @ L1)) - 1).max() < 1e-10 and np.abs(np.exp(1j * (k @ L2)) - 1).max() < 1e-10
        # distinct modulo the reciprocal lattice
        frac = np.stack([k @ a1, k @ a2], axis=1) / (2 * np.pi) % 1.0
        d = np.abs(frac[:, None, :] - frac[None, :, :])
        d = np.minimum(d, 1 - d).max(axis=2)
        assert (d + np.eye(n)).min() > 1e-6


def _cells_honeycomb(L1, L2):
    return np.array([[c % L1, c // L1] for c in range(L1 * L2)], dtype=float)


def test_structure_factor_matches_the_paper_double_sum_with_orbitals():
    """S_ab(k) = (1/N_cell) sum_ij e^{-i k (i - j)} <O_ia O_jb> (Eq. s_corr) with
    a random pair function on a 3 x 2 honeycomb (two orbitals), through the class
    sums of translation_classes_honeycomb."""
    L1, L2 = 3, 2
    ncell = L1 * L2
    N = 2 * ncell
    rng = np.random.default_rng(3)
    M = rng.standard_normal((N, N))
    cls, ncls, r = W.translation_classes_honeycomb(L1, L2)
    C = np.bincount(cls, weights=M.ravel(), minlength=ncls)
    k = A.momenta(A1, A2H, L1 * A1, L2 * A2H)
    S = A.structure_factor(C, r, A1, A2H, k, ncell, n_orb=2)
    cells = _cells_honeycomb(L1, L2)
    pos = cells[:, :1] * A1 + cells[:, 1:] * A2H
    for q, kq in enumerate(k):
        for a in range(2):
            for b in range(2):
                direct = sum(np.exp(-1j * kq @ (pos[i] - pos[j])) * M[2 * i + a, 2 * j + b]
                             for i in range(ncell) for j in range(ncell)) / ncell
                assert S[q, a, b] == pytest.approx(direct, abs=1e-12)
    # leading dimensions (bins, tau) are carried through
    S2 = A.structure_factor(np.stack([C, 2 * C]), r, A1, A2H, k, ncell, n_orb=2)
    assert np.abs(S2[0] - S).max() < 1e-13 and np.abs(S2[1] - 2 * S).max() < 1e-12


def test_background_is_subtracted_at_zero_momentum_only():
    L1, L2 = 3, 3
    ncell = L1 * L2
    rng = np.random.default_rng(4)
    cls, ncls, r = W.translation_classes_honeycomb(L1, L2)
    C = rng.standard_normal(ncls)
    k = A.momenta(A1, A2H, L1 * A1, L2 * A2H)
    O = np.array([0.3, -0.7])
    S0 = A.structure_factor(C, r, A1, A2H, k, ncell, n_orb=2)
    S1 = A.structure_factor(C, r, A1, A2H, k, ncell, n_orb=2, O_mean=O)
    diff = S0 - S1
    assert np.abs(diff[0] - ncell * np.outer(O, O)).max() < 1e-13    # k = 0 comes first
    assert np.abs(diff[1:]).max() == 0.0


def _free_green(K, beta):
    w, V = np.linalg.eigh(K)
    return (V / (1.0 + np.exp(-beta * w))) @ V.T                         # G = <c c+> = (1 + e^{-beta K})^-1


def test_free_fermion_momentum_distribution_square():
    """U = 0: the structure factor of sum_s <c+_x c_y> is 2 f(eps_k),
    eps_k = -2 t (cos k_x + cos k_y) - mu (the closed form of the free lattice)."""
    Lx, Ly, t, mu, beta = 4, 4, 1.0, -0.3, 2.0
    K = W.square_lattice(Lx, Ly, t, 0.0, mu)
    G = _free_green(K, beta)
    N = Lx * Ly
    cls, ncls, r = W.translation_classes_square(Lx, Ly)
    pair = 2.0 * (np.eye(N) - G.T)                                        # sum_s <c+_x c_y> = 2 (delta - G_yx)
    C = np.bincount(cls, weights=pair.ravel(), minlength=ncls)
    k = A.momenta([1, 0], [0, 1], [Lx, 0], [0, Ly])
    S = A.structure_factor(C, r, [1, 0], [0, 1], k, N)[:, 0, 0]
    eps = -2 * t * (np.cos(k[:, 0]) + np.cos(k[:, 1])) - mu
    assert np.abs(S - 2.0 / (1.0 + np.exp(beta * eps))).max() < 1e-12


def test_free_fermion_momentum_distribution_honeycomb():
    """U = 0 on the honeycomb: the orbital trace of S_ab(k) for sum_s <c+ c> is
    2 sum_n f(eps_n(k)) over the two bands of the Bloch Hamiltonian, and S(k) is
    Hermitian."""
    L1, L2, t, mu, beta = 3, 3, 1.0, 0.2, 3.0
    ncell = L1 * L2
    N = 2 * ncell
    K = W.honeycomb_lattice(L1, L2, t, mu)
    G = _free_green(K, beta)
    cls, ncls, r = W.translation_classes_honeycomb(L1, L2)
    C = np.bincount(cls, weights=(2.0 * (np.eye(N) - G.T)).ravel(), minlength=ncls)
    k = A.momenta(A1, A2H, L1 * A1, L2 * A2H)
    S = A.structure_factor(C, r, A1, A2H, k, ncell, n_orb=2)
    cells = _cells_honeycomb(L1, L2)
    pos = cells[:, :1] * A1 + cells[:, 1:] * A2H
    for q, kq in enumerate(k):
        H = np.zeros((2, 2), dtype=complex)                               # Bloch Hamiltonian from cell 0
        for j in range(ncell):
            H += K[0:2, 2 * j:2 * j + 2] * np.exp(1j * kq @ pos[j])
        eps = np.linalg.eigvalsh(H)
        assert np.trace(S[q]).real == pytest.approx(2.0 * np.sum(1.0 / (1.0 + np.exp(beta * eps))), abs=1e-12)
        assert abs(np.trace(S[q]).imag) < 1e-12
        assert np.abs(S[q] - S[q].conj().T).max() < 1e-12


def test_obser_latt_jackknife():
    L1, L2 = 2, 2
    ncell = L1 * L2
    cls, ncls, r = W.translation_classes_honeycomb(L1, L2)
    k = A.momenta(A1, A2H, L1 * A1, L2 * A2H)
    rng = np.random.default_rng(6)
    C = rng.standard_normal(ncls)
    O = rng.standard_normal(2)
    # identical bins: no spread, and the estimate of the pooled ratio
    mean, er, ei = A.obser_latt(np.tile(C, (5, 1)) * 0.5, np.full(5, 0.5), r, A1, A2H, k, ncell, 2,
                                O_sign=np.tile(O, (5, 1)) * 0.5)
    assert np.abs(mean - A.structure_factor(C, r, A1, A2H, k, ncell, 2, O_mean=O)).max() < 1e-12
    assert er.max() < 1e-12 and ei.max() < 1e-12
    # sign-reweighted bins: the mean of the leave-one-bin-out structure factors (Eq. jack_mean)
    s = np.where(rng.random(20) < 0.8, 1.0, -1.0) * (0.5 + rng.random(20))
    Cb = rng.standard_normal((20, ncls)) * s[:, None]
    mean, er, ei = A.obser_latt(Cb, s, r, A1, A2H, k, ncell, 2)
    loo = np.array([A.structure_factor((Cb.sum(0) - Cb[i]) / (s.sum() - s[i]), r, A1, A2H, k, ncell, 2)
                    for i in range(20)])
    assert np.abs(mean - loo.mean(axis=0)).max() < 1e-12
    assert np.abs(er - np.sqrt(19 / 20 * ((loo.real - loo.real.mean(0)) ** 2).sum(0))).max() < 1e-12
    assert er.max() > 0 and np.isfinite(er).all() and np.isfinite(ei).all()
    with pytest.raises(ValueError):
        A.obser_latt(Cb[:1], s[:1], r, A1, A2H, k, ncell, 2)


def test_covariance_between_imaginary_times():
    """N_Cov: for plain means (unit signs) the jackknife covariance of S(k, tau)
    is the paper's (1/N_bin) <(S(tau) - <S>)(S(tau') - <S>)> over bins, with the
    bin average bias-corrected (1/(N_bin - 1)) as in the jackknife error, so its
    diagonal is the squared error."""
    L1, L2, n_tau, nb = 2, 2, 3, 12
    ncell = L1 * L2
    cls, ncls, r = W.translation_classes_honeycomb(L1, L2)
    k = A.momenta(A1, A2H, L1 * A1, L2 * A2H)
    rng = np.random.default_rng(8)
    base = rng.standard_normal((n_tau + 1, ncls))
    Cb = base[None] + 0.1 * rng.standard_normal((nb, 1, ncls)) + 0.05 * rng.standard_normal((nb, n_tau + 1, ncls))
    mean, er, ei, cov = A.obser_latt(Cb, np.ones(nb), r, A1, A2H, k, ncell, 2, cov=True)
    Sb = A.structure_factor(Cb, r, A1, A2H, k, ncell, 2).real            # per bin [nb, tau, k, a, b]
    dev = Sb - Sb.mean(axis=0)
    want = np.einsum("itkab,iukab->tukab", dev, dev) / nb / (nb - 1)      # covariance of the bin mean
    assert np.abs(cov - want).max() < 1e-12 * max(1.0, np.abs(want).max())
    assert np.abs(np.einsum("ttkab->tkab", cov) - er ** 2).max() < 1e-12
    assert np.abs(mean.real - Sb.mean(axis=0)).max() < 1e-12
    with pytest.raises(ValueError):
        A.obser_latt(Cb[:, 0], np.ones(nb), r, A1, A2H, k, ncell, 2, cov=True)


def test_skip_and_rebin():
    x = np.arange(11.0)
    assert np.array_equal(A.skip_and_rebin(x, n_skip=2, n_rebin=3), np.array([3.0, 6.0, 9.0]))
    assert np.array_equal(A.skip_and_rebin(x), x)
    with pytest.raises(ValueError):
        A.skip_and_rebin(x, n_skip=11)
    with pytest.raises(ValueError):
        A.skip_and_rebin(x, n_rebin=0)
