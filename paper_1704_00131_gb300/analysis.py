"""Host-side analysis of the Monte Carlo measurements (plain numpy).

* `fourier`: lattice Fourier transform of a correlation collected per
  displacement class, S(q) = (1/N) sum_r e^{i q.r} C(r) with C(r) the sum over
  the pairs of the class (the R -> K transform the paper's analysis programs
  apply to Obser_Latt data, Sec. 5.3).
* `rebin` and `jackknife`: error bars of sign-weighted averages
  <O> = <O s> / <s> from per-sample data, as the paper's bin analysis does
  (Sec. 5.3: bins of measurements, then jackknife over bins for ratios).
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
    """Sign-reweighted mean <O> = sum(O s) / sum(s) and its jackknife error.
    obs_sign: per-bin means of O * s, shape [n_bins, ...]; sign: per-bin means of s."""
    os_ = np.asarray(obs_sign, dtype=np.float64)
    s = np.asarray(sign, dtype=np.float64)
    n = s.shape[0]
    if n < 2:
        raise ValueError("need at least two bins")
    sh = (n,) + (1,) * (os_.ndim - 1)
    tot_o, tot_s = os_.sum(axis=0), s.sum()
    mean = tot_o / tot_s
    loo = (tot_o[None] - os_) / (tot_s - s).reshape(sh)          # leave-one-out estimates
    err = np.sqrt((n - 1) / n * ((loo - loo.mean(axis=0)) ** 2).sum(axis=0))
    return mean, err
