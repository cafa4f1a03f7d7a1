"""Pins of the oracle's time-displaced correlation functions per pair class
(orc_tau_correlations: sum_s <c_xs(tau) c^+_ys(0)>, <S^z_x(tau) S^z_y(0)>,
<n_x(tau) n_y(0)> summed over the pairs of each class).

* Exact enumeration of all Ising fields of a dimer and of a 2 x 2 plaquette,
  weighted by det(1 + B_up) det(1 + B_dn), equals the Fock-space trace with the
  operators inserted between the Trotter factors, for every tau and class.
* tau = 0 per configuration: the Green function, S^z S^z and n n sums equal the
  equal-time ones (orc_correlations on the same G; the Green function as
  sum_s G^s_xy of the equal-time G).
* U = 0: closed form of every class sum through the eigenvectors of K (numpy
  eigh): G(tau,0) = e^{-tau dtau K}(1 + e^{-beta K})^-1, G(0,tau) =
  -(1 - G)e^{tau dtau K}, densities from G.
* One configuration at small beta, one class per ordered pair: every entry
  equals the plain numpy product (B_tau = e^{-dtau K} e^{V_tau}, G(tau,0) =
  B(tau,0)(1 + B(beta,0))^-1, G(0,tau) = -(1 - G(0)) B(tau,0)^-1, G(tau,tau) =
  (1 + B(tau,0) B(beta,tau))^-1) on a lattice without inversion symmetry.
* Particle-number conservation per configuration: with one class holding every
  pair, sum_xy <n_x(tau) n_y(0)> does not depend on tau.
"""
import itertools
import math

import numpy as np
import pytest

from paper_1704_00131_gb300 import workloads as W

from .fock_ed import Fock, tau_correlations


def make_model(orc, K, U, dtau, L, nwrap):
    N = K.shape[-1]
    sign = np.stack([np.ones(N), -np.ones(N)])
    return orc.Model(np.stack([K, K]), np.arange(N, dtype=np.int32), sign, U, dtau, L, nwrap, 1)


@pytest.mark.parametrize("cluster", ["dimer", "plaquette"])
def test_enumeration_equals_fock_trace(orc, cluster):
    if cluster == "dimer":
        K, U, dtau, L = W.chain_lattice(2, t=1.0, mu=0.3), 3.0, 0.25, 4
        cls, ncls = np.array([0, 1, 1, 0], dtype=np.int32), 2
    else:
        K, U, dtau, L = W.square_lattice(2, 2, t=1.0, mu=0.2), 4.0, 0.3, 3
        cls, ncls, _ = W.translation_classes_square(2, 2)
    N = K.shape[0]
    m = make_model(orc, K, U, dtau, L, L)
    Z, acc = 0.0, 0.0
    for bits in itertools.product((-1, 1), repeat=N * L):
        f = np.array(bits, dtype=np.int8).reshape(L, N)
        _, ld0, s0 = orc.green_udv(m, f, 0, 0)
        _, ld1, s1 = orc.green_udv(m, f, 1, 0)
        w = s0 * s1 * math.exp(ld0 + ld1)
        Z += w
        acc = acc + w * orc.tau_correlations(m, f, L, cls, ncls)
    ref = tau_correlations(Fock(N), K, U, dtau, L, cls, ncls)
    assert acc / Z == pytest.approx(ref, rel=1e-10, abs=1e-12)


def test_equal_time_limit(orc):
    K = W.square_lattice(4, 4, t=1.0, tp=-0.2, mu=0.1)
    m = make_model(orc, K, 5.0, 0.1, 20, 5)
    f = W.random_fields(1, 20, 16, seed=8)
    cls, ncls, _ = W.translation_classes_square(4, 4)
    out = orc.tau_correlations(m, f, 0, cls, ncls)
    G = np.stack([orc.green_udv(m, f, s, 0)[0] for s in (0, 1)])
    eq = orc.correlations(G, cls, ncls)
    gsum = np.zeros(ncls)
    np.add.at(gsum, cls, (G[0] + G[1]).ravel())
    assert np.abs(out[0, :, 0] - gsum).max() < 1e-12
    assert np.abs(out[0, :, 1] - eq[:, 0]).max() < 1e-12
    assert np.abs(out[0, :, 2] - eq[:, 1]).max() < 1e-12


def test_free_closed_form(orc):
    K = W.square_lattice(4, 2, t=1.0, tp=0.15, mu=-0.3)
    N, L, dtau = 8, 10, 0.1
    m = make_model(orc, K, 0.0, dtau, L, 5)
    f = W.random_fields(1, L, N, seed=2)
    cls, ncls, _ = W.translation_classes_square(4, 2)
    out = orc.tau_correlations(m, f, L, cls, ncls)
    w, V = np.linalg.eigh(K)
    G = (V / (1.0 + np.exp(-L * dtau * w))) @ V.T
    n = 1.0 - np.diag(G)
    for tau in range(L + 1):
        Et = (V * np.exp(-tau * dtau * w)) @ V.T
        Gt0 = Et @ G
        G0t = -(np.eye(N) - G) @ np.linalg.inv(Et)
        X = -G0t.T * Gt0                              # X_xy = -G(0,tau)_yx G(tau,0)_xy, per flavor
        want = np.zeros((ncls, 3))
        for x in range(N):
            for y in range(N):
                c = cls[x * N + y]
                want[c, 0] += 2 * Gt0[x, y]
                want[c, 1] += 0.25 * 2 * X[x, y]      # spin-symmetric at U = 0: m_x = 0
                want[c, 2] += 4 * n[x] * n[y] + 2 * X[x, y]
        assert np.abs(out[tau] - want).max() < 1e-11, tau


def test_total_density_correlation_is_tau_independent(orc):
    K = W.chain_lattice(6, t=1.0, mu=0.4, periodic=True)
    m = make_model(orc, K, 4.0, 0.125, 16, 4)
    f = W.random_fields(1, 16, 6, seed=5)
    cls = np.zeros(36, dtype=np.int32)
    out = orc.tau_correlations(m, f, 16, cls, 1)
    assert np.abs(out[:, 0, 2] - out[0, 0, 2]).max() < 1e-9


def test_single_configuration_against_plain_products(orc):
    from scipy.linalg import expm
    K = W.chain_lattice(4, t=1.0, mu=0.2)
    K[0, 0] -= 0.3
    K[1, 3] = K[3, 1] = -0.4
    N, U, dtau, L = 4, 4.0, 0.1, 6
    m = make_model(orc, K, U, dtau, L, 3)
    f = W.random_fields(1, L, N, seed=12).reshape(L, N)
    out = orc.tau_correlations(m, f, L, np.arange(N * N, dtype=np.int32), N * N)
    lam = np.arccosh(np.exp(0.5 * dtau * U))
    E = expm(-dtau * K)
    I = np.eye(N)
    Gt0, G0t, Gtt = {}, {}, {}
    for s, sig in ((0, 1.0), (1, -1.0)):
        Bs = [E @ np.diag(np.exp(sig * lam * f[t].astype(float))) for t in range(L)]
        def prod(a, b):                               # B(a, b) = B_a ... B_{b+1}
            P = I.copy()
            for t in range(b, a):
                P = Bs[t] @ P
            return P
        G0 = np.linalg.inv(I + prod(L, 0))
        for tau in range(L + 1):
            Gt0[s, tau] = prod(tau, 0) @ G0
            G0t[s, tau] = -(I - G0) @ np.linalg.inv(prod(tau, 0))
            Gtt[s, tau] = np.linalg.inv(I + prod(tau, 0) @ prod(L, tau))
    for tau in range(L + 1):
        want = np.zeros((N, N, 3))
        m_t = (1 - np.diag(Gtt[0, tau])) - (1 - np.diag(Gtt[1, tau]))
        r_t = (1 - np.diag(Gtt[0, tau])) + (1 - np.diag(Gtt[1, tau]))
        m_0 = (1 - np.diag(Gtt[0, 0])) - (1 - np.diag(Gtt[1, 0]))
        r_0 = (1 - np.diag(Gtt[0, 0])) + (1 - np.diag(Gtt[1, 0]))
        X = sum(-G0t[s, tau].T * Gt0[s, tau] for s in (0, 1))
        want[..., 0] = Gt0[0, tau] + Gt0[1, tau]
        want[..., 1] = 0.25 * (np.outer(m_t, m_0) + X)
        want[..., 2] = np.outer(r_t, r_0) + X
        assert np.abs(out[tau].reshape(N, N, 3) - want).max() < 1e-11, tau
