"""Host-side analysis of the Monte Carlo measurements (plain numpy).

* `fourier`: lattice Fourier transform of a correlation collected per
  displacement class, S(q) = (1/N) sum_r e^{i q.r} C(r) with C(r) the sum over
  the pairs of the class (the R -> K transform the paper's analysis programs
  apply to Obser_Latt data, Sec. 5.3).
* `rebin`, `skip_and_rebin` and `jackknife`: error bars of sign-weighted
  averages <O> = <O s> / <s> from per-bin data, as the paper's bin analysis
  does (Sec. 5.3: n_skip and N_rebin, then the delete-1 jackknife over bins,
  Eqs. jack_mean and jack_error).
* `reciprocal_vectors`, `k_quantisation`, `momenta`: the momentum grid of a
  periodic Bravais lattice with unit vectors a_1, a_2 and periodicity vectors
  L_1, L_2 (Sec. 3.2, the Lattice type: a_i . g_j = 2 pi delta_ij and the
  quantisation k = n b_1 + m b_2 of Eq. k.quant; tilted lattices included).
* `structure_factor` and `obser_latt`: the orbital-resolved correlation
  function S_ab(k, tau) of an Obser_Latt observable (Sec. 5.1, Eq. s with its
  correlated part s_corr and background part s_back) from per-class sums of a
  multi-orbital lattice, and its sign-reweighted jackknife over bins.
"""
from __future__ import annotations

import numpy as np


def momenta_square(Lx: int, Ly: int) -> np.ndarray:
    """The Lx * Ly momenta (2 pi nx / Lx, 2 pi ny / Ly) of the periodic square lattice."""
    return np.array([[2 * np.pi * nx / Lx, 2 * np.pi * ny / Ly] for ny in range(Ly) for nx in range(Lx)])


def fourier(C: np.ndarray, r: np.ndarray, q: np.ndarray, n_sites: int) -> np.ndarray:
    """S(q) = (1/N) sum_k e^{i q . r_k} C_k for classes k with displacement r_k.
    C: [..., n_class]; r: [n_class, d]; q: [n_q, d].  Returns [..., n_q] (complex)."""
    phase = np.exp(1j * (np.asarray(q) @ np.asarray(r).T))        # [n_q, n_class]
    return np.asarray(C) @ phase.T / float(n_sites)


def rebin(x: np.ndarray, n_bins: int) -> np.ndarray:
    """Means of n_bins consecutive equal-size bins along axis 0 (the tail that
    does not fill a bin is dropped)."""
    x = np.asarray(x, dtype=np.float64)
    size = x.shape[0] // n_bins
    if size < 1:
        raise ValueError("fewer samples than bins")
    return x[: size * n_bins].reshape(n_bins, size, *x.shape[1:]).mean(axis=1)


def jackknife(obs_sign: np.ndarray, sign: np.ndarray):
    """Sign-reweighted <O> = <O s> / <s> by the delete-1 jackknife over bins
    (Sec. 5.3): with f_(i) the ratio of the means without bin i, the estimate is
    f_(.) = (1/N) sum_i f_(i) (Eq. jack_mean) and its error
    sqrt((N-1)/N sum_i (f_(i) - f_(.))^2) (Eq. jack_error).
    obs_sign: per-bin means of O * s, shape [n_bins, ...]; sign: per-bin means of s."""
    os_ = np.asarray(obs_sign, dtype=np.float64)
    s = np.asarray(sign, dtype=np.float64)
    n = s.shape[0]
    if n < 2:
        raise ValueError("need at least two bins")
    sh = (n,) + (1,) * (os_.ndim - 1)
    tot_o, tot_s = os_.sum(axis=0), s.sum()
    loo = (tot_o[None] - os_) / (tot_s - s).reshape(sh)          # f_(i)
    mean = loo.mean(axis=0)                                        # f_(.)
    err = np.sqrt((n - 1) / n * ((loo - mean) ** 2).sum(axis=0))
    return mean, err


def skip_and_rebin(bins: np.ndarray, n_skip: int = 0, n_rebin: int = 1) -> np.ndarray:
    """The analysis parameters n_skip and N_rebin of Sec. 5.3: drop the first
    n_skip bins (warm-up), then merge every n_rebin consecutive bins into one
    (their mean; a tail that does not fill a merged bin is dropped)."""
    b = np.asarray(bins, dtype=np.float64)
    if n_skip < 0 or n_rebin < 1:
        raise ValueError("need n_skip >= 0 and n_rebin >= 1")
    b = b[n_skip:]
    m = b.shape[0] // n_rebin
    if m < 1:
        raise ValueError("no bins left after n_skip and n_rebin")
    return b[: m * n_rebin].reshape((m, n_rebin) + b.shape[1:]).mean(axis=1)


def reciprocal_vectors(a1, a2):
    """g_1, g_2 with a_i . g_j = 2 pi delta_ij (two dimensions)."""
    A = np.array([a1, a2], dtype=np.float64)
    G = 2.0 * np.pi * np.linalg.inv(A).T          # rows g_j: A @ G.T = 2 pi 1
    return G[0], G[1]


def k_quantisation(L1, L2, g1, g2):
    """b_1, b_2 of the momentum grid k = n b_1 + m b_2 allowed by the periodicity
    vectors L_1, L_2 (e^{i k . L_i} = 1), as the paper writes them:
        b_1 = 2 pi [(L_2.g_2) g_1 - (L_2.g_1) g_2] / D,
        b_2 = 2 pi [(L_1.g_1) g_2 - (L_1.g_2) g_1] / D,
        D = (L_1.g_1)(L_2.g_2) - (L_1.g_2)(L_2.g_1)."""
    L1, L2, g1, g2 = (np.asarray(v, dtype=np.float64) for v in (L1, L2, g1, g2))
    d = (L1 @ g1) * (L2 @ g2) - (L1 @ g2) * (L2 @ g1)
    b1 = 2.0 * np.pi / d * ((L2 @ g2) * g1 - (L2 @ g1) * g2)
    b2 = 2.0 * np.pi / d * ((L1 @ g1) * g2 - (L1 @ g2) * g1)
    return b1, b2


def momenta(a1, a2, L1, L2) -> np.ndarray:
    """The N_unit_cell momenta of the lattice: one k = n b_1 + m b_2 per class
    modulo the reciprocal lattice, the smallest (m, n) in lexicographic order
    representing each class (for L_1 = l_1 a_1, L_2 = l_2 a_2 the cell-index
    order n + l_1 m of `translation_classes_square`).  Returns [N_unit_cell, 2]."""
    a1, a2, L1, L2 = (np.asarray(v, dtype=np.float64) for v in (a1, a2, L1, L2))
    n_cells = int(round(abs(np.linalg.det(np.array([L1, L2]))) / abs(np.linalg.det(np.array([a1, a2])))))
    g1, g2 = reciprocal_vectors(a1, a2)
    b1, b2 = k_quantisation(L1, L2, g1, g2)
    m, n = np.meshgrid(np.arange(n_cells), np.arange(n_cells), indexing="ij")
    ks = n.reshape(-1, 1) * b1 + m.reshape(-1, 1) * b2
    frac = np.stack([ks @ a1, ks @ a2], axis=1) / (2.0 * np.pi)     # k in units of g_1, g_2
    key = np.round((frac % 1.0) * 1e8).astype(np.int64) % 100000000
    _, first = np.unique(key, axis=0, return_index=True)
    first = np.sort(first)
    if first.size != n_cells:
        raise ValueError(f"found {first.size} momenta for {n_cells} unit cells")
    return ks[first]


def _is_zero_momentum(k, a1, a2) -> np.ndarray:
    frac = np.stack([np.asarray(k) @ np.asarray(a1, float), np.asarray(k) @ np.asarray(a2, float)], axis=-1)
    frac = frac / (2.0 * np.pi)
    return np.all(np.abs(frac - np.round(frac)) < 1e-9, axis=-1)


def structure_factor(C, r_cells, a1, a2, k, n_cells: int, n_orb: int = 1, O_mean=None) -> np.ndarray:
    """S_ab(k) = (1/N_cell) sum_d e^{i k . R_d} C(d, a, b) - N_cell <O_a><O_b> delta(k).

    C: [..., n_class] sums of <O_x O_y> over the pairs of each class, classes
    ordered as n_orb^2 d + n_orb a + b for the cell displacement d = cell(y) -
    cell(x) and orbitals a of x, b of y (as `translation_classes_square` and
    `translation_classes_honeycomb` number them); leading dimensions (bins,
    tau) are kept.  With x = (i, a), y = (j, b) the phase e^{i k . R_d} is the
    paper's e^{-i k . (i - j)} (Eq. s_corr).  r_cells: [n_class, 2] cell
    displacement of each class in units of a_1, a_2.  k: [n_k, 2].
    O_mean: [..., n_orb] the per-orbital means <O_a> = (1/N_cell) sum_i <O_ia>
    (Eq. o); when given, the background N_cell <O_a><O_b> at k = 0 (Eq. s_back)
    is subtracted.  Returns [..., n_k, n_orb, n_orb] complex."""
    C = np.asarray(C)
    no2 = n_orb * n_orb
    if C.shape[-1] % no2:
        raise ValueError("the number of classes is not a multiple of n_orb^2")
    n_d = C.shape[-1] // no2
    R = np.asarray(r_cells, dtype=np.float64).reshape(n_d, no2, 2)[:, 0, :]
    Rv = R[:, :1] * np.asarray(a1, float) + R[:, 1:2] * np.asarray(a2, float)   # [n_d, 2]
    phase = np.exp(1j * (np.asarray(k, dtype=np.float64) @ Rv.T))                # [n_k, n_d]
    Cd = C.reshape(C.shape[:-1] + (n_d, n_orb, n_orb))
    S = np.einsum("kd,...dab->...kab", phase, Cd) / float(n_cells)
    if O_mean is not None:
        O = np.asarray(O_mean)
        back = float(n_cells) * O[..., :, None] * O[..., None, :]                 # [..., n_orb, n_orb]
        zero = _is_zero_momentum(k, a1, a2)
        S = S - zero[:, None, None] * back[..., None, :, :]
    return S


def obser_latt(C_sign, sign, r_cells, a1, a2, k, n_cells: int, n_orb: int = 1, O_sign=None, cov: bool = False):
    """Bin analysis of an Obser_Latt observable (Sec. 5.1 and 5.3): from the
    per-bin means of the sign-weighted class sums C s ([n_bins, ..., n_class]),
    of the sign s ([n_bins]) and optionally of the sign-weighted per-orbital
    means O s ([n_bins, ..., n_orb]), the structure factor S_ab(k) of <C s>/<s>
    with the background of <O s>/<s>, by the delete-1 jackknife over bins: the
    mean of the leave-one-bin-out estimates f_(i) and the error
    sqrt((N-1)/N sum_i (f_(i) - f_(.))^2), real and imaginary parts separately.
    Returns (mean, err_re, err_im), each [..., n_k, n_orb, n_orb]; with cov and a
    leading tau axis (C_sign [n_bins, n_tau, n_class]) also the covariance of
    Re S between imaginary times (the N_Cov option of Sec. 5.3),
    COV[t, t'] = (N-1)/N sum_i (f_(i)(t) - f_(.)(t)) (f_(i)(t') - f_(.)(t')),
    [n_tau, n_tau, n_k, n_orb, n_orb]; its diagonal is err_re^2, and for a
    plain mean it is the paper's (1/N_bin) <(S(t) - <S(t)>)(S(t') - <S(t')>)>
    with the average over bins taken with the bias correction of Eq. jack_error
    (1/(N_bin - 1)), so that the diagonal is the squared jackknife error."""
    Cs = np.asarray(C_sign, dtype=np.float64)
    s = np.asarray(sign, dtype=np.float64)
    n = s.shape[0]
    if n < 2:
        raise ValueError("need at least two bins")
    Os = None if O_sign is None else np.asarray(O_sign, dtype=np.float64)

    def estimate(csum, osum, ssum):
        return structure_factor(csum / ssum, r_cells, a1, a2, k, n_cells, n_orb,
                                None if osum is None else osum / ssum)

    tot_c, tot_s = Cs.sum(axis=0), s.sum()
    tot_o = None if Os is None else Os.sum(axis=0)
    loo = np.stack([estimate(tot_c - Cs[b], None if Os is None else tot_o - Os[b], tot_s - s[b])
                    for b in range(n)])                                     # f_(i)
    mean = loo.mean(axis=0)                                                  # f_(.)
    dev = loo - mean
    f = (n - 1) / n
    out = (mean, np.sqrt(f * (dev.real ** 2).sum(axis=0)), np.sqrt(f * (dev.imag ** 2).sum(axis=0)))
    if cov:
        if Cs.ndim != 3:
            raise ValueError("cov needs C_sign of shape [n_bins, n_tau, n_class]")
        d = dev.real                                                         # [n_bins, n_tau, n_k, a, b]
        out = out + (f * np.einsum("itkab,iukab->tukab", d, d),)
    return out
