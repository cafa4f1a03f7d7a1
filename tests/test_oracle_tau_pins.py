"""Pins of the oracle's time-displaced measurement (orc_tau_observables).

* U = 0: every Green function has a closed form through the eigenvectors of K,
  G(tau,0) = e^{-tau dtau K} (1 + e^{-beta K})^-1, G(0,tau) = -(1 - G) e^{tau dtau K},
  G(tau,tau) = G (numpy eigh, not the oracle's Jacobi).
* Anti-periodicity at tau = L: G(beta,0) = 1 - G(0) and G(0,beta) = -G(0).
* Particle-number conservation per flavor: with unit phases, p_s(tau) and the
  connected sum c_s(tau) do not depend on tau in any configuration.
* Exact enumeration of all Ising fields of a dimer and a three-site chain,
  weighted by det(1 + B_up) det(1 + B_dn), equals the Fock-space trace with the
  operators inserted between the Trotter factors:
  <A(tau) B(0)> = Tr[T^{L-tau} A T^tau B] / Tr[T^L], T = e^{-dtau H_T} e^{-dtau H_U}.
"""
import itertools
import math

import numpy as np
import pytest

from paper_1704_00131_gb300 import workloads as W

from .fock_ed import Fock, hs4_slice, tau_observables


def make_model(orc, K, U, dtau, L, nwrap, ft=1):
    N = K.shape[-1]
    sign = np.stack([np.ones(N), -np.ones(N)])
    return orc.Model(np.stack([K, K]), np.arange(N, dtype=np.int32), sign, U, dtau, L, nwrap, ft)


def test_tau_observables_free_closed_form(orc):
    K = W.square_lattice(4, 4, t=1.0, tp=-0.2, mu=-0.4)
    N, L, dtau = 16, 12, 0.1
    ph = W.sublattice_signs_square(4, 4)
    m = make_model(orc, K, 0.0, dtau, L, 4)
    f = W.random_fields(1, L, N, seed=3)
    out, sg = orc.tau_observables(m, f, L, ph)
    w, V = np.linalg.eigh(K)
    G = (V / (1.0 + np.exp(-L * dtau * w))) @ V.T
    for tau in range(L + 1):
        Gt0 = (V * np.exp(-tau * dtau * w)) @ V.T @ G
        G0t = -(np.eye(N) - G) @ ((V * np.exp(tau * dtau * w)) @ V.T)
        a = np.trace(Gt0)
        c = -np.einsum("x,y,yx,xy->", ph, ph, G0t, Gt0)
        p = np.sum(ph * (1.0 - np.diag(G)))
        for s in range(2):
            assert out[tau, s] == pytest.approx([a, c, p], rel=1e-10, abs=1e-10), (tau, s)
    assert list(sg) == [1, 1]


def test_displaced_green_antiperiodic_at_beta(orc):
    K = W.square_lattice(4, 4)
    L = 20
    m = make_model(orc, K, 4.0, 0.1, L, 5)
    f = W.random_fields(1, L, 16, seed=9)
    for s in (0, 1):
        G0, _, _ = orc.green_udv(m, f, s, 0)
        Gt0, G0t = orc.green_displaced(m, f, s, L)
        assert np.abs(Gt0 - (np.eye(16) - G0)).max() < 1e-10
        assert np.abs(G0t + G0).max() < 1e-10
        # tau = 0: G(0,0) = G(0), G(0,0^+) = -(1 - G(0))
        Gt0, G0t = orc.green_displaced(m, f, s, 0)
        assert np.abs(Gt0 - G0).max() < 1e-12
        assert np.abs(G0t + (np.eye(16) - G0)).max() < 1e-12


def test_conserved_particle_number_per_configuration(orc):
    K = W.honeycomb_lattice(2, 2)
    N, L = K.shape[0], 16
    m = make_model(orc, K, 5.0, 0.125, L, 4)
    f = W.random_fields(1, L, N, seed=21)
    out, _ = orc.tau_observables(m, f, L)
    for s in (0, 1):
        assert np.ptp(out[:, s, 2]) < 1e-10   # N_s
        assert np.ptp(out[:, s, 1]) < 1e-10   # connected <N_s(tau) N_s(0)>
    # a staggered phase does not commute with H: the sums must move
    ph = np.where(np.arange(N) % 2 == 0, 1.0, -1.0)
    out2, _ = orc.tau_observables(m, f, L, ph)
    assert np.ptp(out2[:, 0, 1]) > 1e-3


@pytest.mark.parametrize("cluster", ["dimer", "chain3"])
def test_tau_enumeration_equals_fock_trace(orc, cluster):
    if cluster == "dimer":
        K, U, dtau, L = W.chain_lattice(2, t=1.0, mu=0.3), 3.0, 0.25, 4
        ph = np.array([1.0, -1.0])
    else:
        K, U, dtau, L = W.chain_lattice(3, t=1.0, mu=-0.2, periodic=False), 4.0, 0.3, 3
        ph = np.array([1.0, -1.0, 1.0])
    N = K.shape[0]
    m = make_model(orc, K, U, dtau, L, L)
    Z = 0.0
    gl = np.zeros(L + 1)
    szz = np.zeros(L + 1)
    for bits in itertools.product((-1, 1), repeat=N * L):
        f = np.array(bits, dtype=np.int8).reshape(L, N)
        _, ld0, s0 = orc.green_udv(m, f, 0, 0)
        _, ld1, s1 = orc.green_udv(m, f, 1, 0)
        w = s0 * s1 * math.exp(ld0 + ld1)
        out, sg = orc.tau_observables(m, f, L, ph)
        assert sg[0] == s0 and sg[1] == s1
        Z += w
        gl += w * (out[:, 0, 0] + out[:, 1, 0])
        szz += w * orc.szz_from_tau(out)
    F = Fock(N)
    gl_ed, szz_ed = tau_observables(F, K, U, dtau, L, ph)
    assert gl / Z == pytest.approx(gl_ed, rel=1e-10, abs=1e-12)
    assert szz / Z == pytest.approx(szz_ed, rel=1e-10, abs=1e-12)


def test_tau_enumeration_equals_fock_trace_hs4(orc):
    """Four-valued HS fields of a dimer (4^(N L) = 4096 configurations), weighted
    by prod gamma(l)/4 and the determinants: the time-displaced averages equal the
    Fock trace with the summed HS4 slice factor inserted between hoppings."""
    K, U, dtau, L = W.chain_lattice(2, t=1.0, mu=-0.2), 4.0, 0.2, 3
    N = 2
    ph = np.array([1.0, -1.0])
    m = make_model(orc, K, U, dtau, L, L, ft=2)
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}
    eta = {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)}
    Z = 0.0
    gl = np.zeros(L + 1)
    szz = np.zeros(L + 1)
    for ls in itertools.product((-2, -1, 1, 2), repeat=N * L):
        f = np.array(ls, dtype=np.int8).reshape(L, N)
        _, ld0, s0 = orc.green_udv(m, f, 0, 0)
        _, ld1, s1 = orc.green_udv(m, f, 1, 0)
        w = np.prod([gam[l] / 4.0 for l in ls]) * s0 * s1 * math.exp(ld0 + ld1)
        out, _ = orc.tau_observables(m, f, L, ph)
        Z += w
        gl += w * (out[:, 0, 0] + out[:, 1, 0])
        szz += w * orc.szz_from_tau(out)
    F = Fock(N)
    gl_ed, szz_ed = tau_observables(F, K, U, dtau, L, ph, W=hs4_slice(F, U, dtau, eta, gam))
    assert gl / Z == pytest.approx(gl_ed, rel=1e-10, abs=1e-12)
    assert szz / Z == pytest.approx(szz_ed, rel=1e-10, abs=1e-12)
