"""Pins of the oracle's SU(2) charge decoupling with complex coupling
(orc_su2_plain: fixed fields, plain product, two colors).

* Exact enumeration of all four-valued fields of small clusters, each weighted
  by prod gamma/4, the phase exp(-i g sum eta) and det(1 + B)^2, equals the
  Fock-space trace of the Trotter product with the summed slice factor
  W = prod_i sum_l gamma(l)/4 exp(i g eta(l) (n_i - 1)): the partition
  function (its imaginary part cancels) and the energy <H_T + U/2 sum (n_i-1)^2>.
* At half filling on a bipartite lattice every configuration's weight is real
  and positive (no phase problem), away from it the weights are complex.
* U = 0: G = (1 + exp(-beta K))^-1.
"""
import itertools
import math

import numpy as np
import pytest
from scipy.linalg import expm

from paper_1704_00131_gb300 import workloads as W

from .fock_ed import Fock


def su2_fock(K, U, dtau, L, eta, gamma):
    N = K.shape[0]
    F = Fock(N)
    g = math.sqrt(0.5 * dtau * U)
    Wd = np.ones(F.dim, dtype=complex)
    for i in range(N):
        ni = np.diag(F.n(0, i)) + np.diag(F.n(1, i))
        Wd *= sum(gamma[l] / 4.0 * np.exp(1j * g * eta[l] * (ni - 1.0)) for l in (-2, -1, 1, 2))
    T = expm(-dtau * F.hopping(K)) @ np.diag(Wd)
    rho = np.linalg.matrix_power(T, L)
    I = np.eye(F.dim)
    HU = sum(0.5 * U * (F.n(0, i) + F.n(1, i) - I) @ (F.n(0, i) + F.n(1, i) - I) for i in range(N))
    Z = np.trace(rho)
    return Z, np.trace((F.hopping(K) + HU) @ rho) / Z


def enumerate_su2(orc, K, U, dtau, L):
    N = K.shape[0]
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}
    Z, EZ, weights = 0.0, 0.0, []
    for ls in itertools.product((-2, -1, 1, 2), repeat=N * L):
        f = np.array(ls, dtype=np.int8)
        _, la, ar, ph, kin, pot = orc.su2_plain(K, dtau, U, f)
        w = np.prod([gam[l] / 4.0 for l in ls]) * np.exp(1j * ph) * np.exp(2.0 * (la + 1j * ar))
        weights.append(w)
        Z += w
        EZ += w * (kin + pot)
    return Z, EZ / Z, np.array(weights)


@pytest.mark.parametrize("mu", [0.0, 0.4])
def test_su2_enumeration_equals_fock_trace(orc, mu):
    K, U, dtau, L = W.chain_lattice(2, t=1.0, mu=mu), 4.0, 0.25, 3
    eta = {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)}
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}
    Z, E, w = enumerate_su2(orc, K, U, dtau, L)
    Zf, Ef = su2_fock(K, U, dtau, L, eta, gam)
    assert Z == pytest.approx(Zf, rel=1e-11)
    assert abs(Z.imag) < 1e-11 * abs(Z)
    assert E == pytest.approx(Ef, rel=1e-10, abs=1e-12)
    if mu == 0.0:
        assert np.abs(w.imag).max() < 1e-12 * np.abs(w).max() and (w.real > 0).all()
    else:
        assert np.abs(w.imag).max() > 1e-6 * np.abs(w).max()


def test_su2_free_limit(orc):
    K = W.square_lattice(2, 2, t=1.0, mu=0.3)
    dtau, L = 0.1, 10
    f = np.ones(L * 4, dtype=np.int8)
    G, la, ar, ph, kin, pot = orc.su2_plain(K, dtau, 0.0, f)
    w, V = np.linalg.eigh(K)
    Gf = (V / (1.0 + np.exp(-L * dtau * w))) @ V.T
    assert np.abs(G - Gf).max() < 1e-12 and ph == 0.0 and abs(ar) < 1e-12
    assert la == pytest.approx(np.sum(np.log1p(np.exp(-L * dtau * w))), rel=1e-12)
