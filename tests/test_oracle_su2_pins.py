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
* The complex UDV chain (orc_su2_green_udv) equals the plain product where both
  hold (G, log|det|, arg det; G(tau) against the rotated field sequence) and is
  independent of n_wrap at beta = 10.
* Equal-time correlations per pair class (orc_su2_correlations, both colors on
  one complex G): the enumeration of all four-valued fields of a dimer and of a
  three-site chain, weighted as above, equals the Fock trace of S^z S^z, n n,
  S^+ S^- and sum_s c^+ c in the Trotter product, at and away from half filling.
* The oracle's Markov chain, sampled with W = |Re e^{-S}| and reweighted by
  sign e^{-S} / Re e^{-S} (Sec. 2.2), reproduces the energy of the Trotter
  product within 4 sigma, at and away from half filling (the single-
  configuration estimator has heavy tails with the imaginary coupling, so the
  error bar comes from the spread of 32 independent chains).
"""
import itertools
import math

import numpy as np
import pytest

from paper_1704_00131_gb300 import workloads as W

from .fock_ed import Fock, su2_correlations, su2_trotter


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
    Zf, Ef = su2_trotter(Fock(2), K, U, dtau, L, eta, gam)
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


@pytest.mark.parametrize("mu", [0.0, 0.4])
def test_su2_sampler_matches_trotter_energy(orc, mu):
    from paper_1704_00131_gb300 import analysis as A
    K, U, dtau, L = W.chain_lattice(2, t=1.0, mu=mu), 4.0, 0.25, 4
    eta = {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)}
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}
    _, Ef = su2_trotter(Fock(2), K, U, dtau, L, eta, gam)
    n_chains, burn, n = 32, 40, 300
    os_, ss = np.zeros(n_chains, dtype=complex), np.zeros(n_chains)
    acc = 0
    for c in range(n_chains):
        f0 = orc.init_fields(2, L, 2, 11, c)
        ch = orc.Su2Chain(K, dtau, U, f0, seed=11, chain=c)
        for t in range(burn + n):
            o, sg, a = ch.sweep()
            acc += a
            if t >= burn:
                os_[c] += o / n
                ss[c] += sg / n
    assert 0 < acc < n_chains * (burn + n) * 2 * L * 2
    mean_re, err_re = A.jackknife(os_.real, ss)
    mean_im, err_im = A.jackknife(os_.imag, ss)
    assert abs(mean_re - Ef.real) < 4 * err_re
    assert abs(mean_im) < 4 * err_im + 1e-12


def _wrap_angle(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def test_su2_phase_carried_equals_recomputed(orc):
    """The phase P of e^{-S} that the chain carries through its accepted updates
    (P <- P R / |R|, Sec. 2.2 with W = |Re e^{-S}|) equals, after every sweep, the
    phase recomputed from scratch on the chain's fields, exp(i (-g sum eta +
    2 arg det(1 + B))) (both colors).  Away from half filling on a 3-site chain the
    phases are far from real, so a dropped or halved term shows."""
    K, U, dtau, L = W.chain_lattice(3, t=1.0, mu=0.5), 4.0, 0.25, 4
    worst, spread = 0.0, 0.0
    for c in range(4):
        ch = orc.Su2Chain(K, dtau, U, orc.init_fields(2, L, 3, 13, c), seed=13, chain=c)
        for _ in range(5):
            ch.sweep()
            _, _, ar, ph, _, _ = orc.su2_plain(K, dtau, U, ch.fields.reshape(L, 3))
            P = complex(ch.phase[0], ch.phase[1])
            want = np.exp(1j * (ph + 2.0 * ar))
            worst = max(worst, abs(P / abs(P) - want))
            spread = max(spread, abs(np.angle(want)))
    assert worst < 1e-10
    assert spread > 0.3                                  # the pin has power: phases well off the real axis


@pytest.mark.parametrize("lx", [4, 3])
def test_su2_udv_chain_matches_plain_product(orc, lx):
    """The complex UDV chain (QR with pivoting, scale separation) against the plain
    product where both hold (beta = 2): G, log|det| and arg det for several n_wrap,
    and G(tau) against the plain product of the cyclically rotated fields.  The odd
    3 x 3 torus gives a Householder QR of N = 9 reflections, det Q = -1, so the
    factor det Q_R conj(det Q_L) of arg det is exercised (at tau = 0 the right
    chain is the identity)."""
    rng = np.random.default_rng(0)
    K = W.square_lattice(lx, lx, t=1.0, mu=0.2)
    f = rng.choice([-2, -1, 1, 2], size=(20, lx * lx)).astype(np.int8)
    Gp, la, ar, _, _, _ = orc.su2_plain(K, 0.1, 4.0, f)
    for nw in (1, 5, 20):
        Gu, lu, au = orc.su2_green_udv(K, 0.1, 4.0, nw, f, 0)
        assert np.abs(Gu - Gp).max() < 1e-12
        assert lu == pytest.approx(la, rel=1e-12)
        assert abs(_wrap_angle(au - ar)) < 1e-10
    for tau in (3, 7, 20):
        Gt, _, _ = orc.su2_green_udv(K, 0.1, 4.0, 5, f, tau)
        rot = np.concatenate([f[tau:], f[:tau]])
        Gr, _, _, _, _, _ = orc.su2_plain(K, 0.1, 4.0, rot)
        assert np.abs(Gt - Gr).max() < 1e-12, tau


def test_su2_udv_chain_is_independent_of_n_wrap_at_large_beta(orc):
    rng = np.random.default_rng(1)
    K = W.square_lattice(4, 4, t=1.0, mu=0.2)
    f = rng.choice([-2, -1, 1, 2], size=(100, 16)).astype(np.int8)     # beta = 10
    G5, l5, a5 = orc.su2_green_udv(K, 0.1, 4.0, 5, f, 0)
    G10, l10, a10 = orc.su2_green_udv(K, 0.1, 4.0, 10, f, 0)
    assert np.abs(G5 - G10).max() < 1e-10
    assert l5 == pytest.approx(l10, rel=1e-12) and abs(_wrap_angle(a5 - a10)) < 1e-10


@pytest.mark.parametrize("case", ["dimer_half", "dimer_mu", "chain3_mu"])
def test_su2_correlations_enumeration_equals_fock_trace(orc, case):
    if case.startswith("dimer"):
        K, L = W.chain_lattice(2, t=1.0, mu=0.0 if case == "dimer_half" else 0.4), 3
        cls, ncls = np.array([0, 1, 1, 0], dtype=np.int32), 2
    else:
        K, L = W.chain_lattice(3, t=1.0, mu=0.3), 2
        cls, ncls = np.array([0, 1, 2, 1, 0, 1, 2, 1, 0], dtype=np.int32), 3
    U, dtau = 4.0, 0.25
    N = K.shape[0]
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}
    eta = {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)}
    Z, acc = 0.0, 0.0
    for ls in itertools.product((-2, -1, 1, 2), repeat=N * L):
        f = np.array(ls, dtype=np.int8)
        G, la, ar, ph, _, _ = orc.su2_plain(K, dtau, U, f)
        w = np.prod([gam[l] / 4.0 for l in ls]) * np.exp(1j * ph) * np.exp(2.0 * (la + 1j * ar))
        Z += w
        acc = acc + w * orc.su2_correlations(G, cls, ncls)
    ref = su2_correlations(Fock(N), K, U, dtau, L, eta, gam, cls, ncls)
    got = acc / Z
    assert np.abs(got - ref).max() < 1e-10 * max(1.0, np.abs(ref).max())
    assert np.abs(ref.imag).max() < 1e-12 and np.abs(got.imag).max() < 1e-10


def _su2_B(K, dtau, U, fields, orc):
    """B_t = exp(-dtau K) exp(i g eta(l_t)) of every slice, plain numpy."""
    w, V = np.linalg.eigh(K)
    E = (V * np.exp(-dtau * w)) @ V.T
    g = np.sqrt(0.5 * dtau * U)
    eta = {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)}
    return [E * np.exp(1j * g * np.array([eta[int(l)] for l in f]))[None, :] for f in fields]


def test_su2_displaced_green_matches_the_definition(orc):
    """orc_su2_green_displaced (complex UDV chains, scale separation) against the
    definitions G(tau,0) = B(tau,0) G(0) and G(0,tau) = -(1 - G(0)) B(tau,0)^-1
    with plain products and a dense inverse, where both hold (beta = 2), for
    several chunk lengths, at tau = 0 (G(0), -(1 - G(0))) and beyond."""
    rng = np.random.default_rng(3)
    K = W.square_lattice(4, 4, t=1.0, mu=0.2)
    dtau, U, L = 0.1, 4.0, 20
    f = rng.choice([-2, -1, 1, 2], size=(L, 16)).astype(np.int8)
    Bs = _su2_B(K, dtau, U, f, orc)
    I = np.eye(16)
    Bb = I.astype(complex)
    for B in Bs:
        Bb = B @ Bb
    G0 = np.linalg.inv(I + Bb)
    for nw in (1, 5, 20):
        for tau in (0, 3, 7, 20):
            Bt = I.astype(complex)
            for B in Bs[:tau]:
                Bt = B @ Bt
            Gt0, G0t = orc.su2_green_displaced(K, dtau, U, nw, f, tau)
            assert np.abs(Gt0 - Bt @ G0).max() < 1e-10, (nw, tau)
            assert np.abs(G0t + (I - G0) @ np.linalg.inv(Bt)).max() < 1e-10, (nw, tau)


def test_su2_displaced_green_free_limit(orc):
    """U = 0: G(tau,0) = e^{-tau dtau K} (1 + e^{-beta K})^-1 and
    G(0,tau) = -(1 - G(0)) e^{tau dtau K}, in K's eigenbasis."""
    K = W.square_lattice(4, 4, t=1.0, mu=-0.3)
    dtau, L = 0.1, 60
    w, V = np.linalg.eigh(K)
    f = np.ones((L, 16), dtype=np.int8)
    for tau in (0, 13, 60):
        Gt0, G0t = orc.su2_green_displaced(K, dtau, 0.0, 10, f, tau)
        nk = 1.0 / (1.0 + np.exp(-L * dtau * w))
        hk = 1.0 / (1.0 + np.exp(L * dtau * w))      # 1 - n_k without cancellation
        assert np.abs(Gt0 - (V * (np.exp(-tau * dtau * w) * nk)) @ V.T).max() < 1e-12
        assert np.abs(G0t + (V * (hk * np.exp(tau * dtau * w))) @ V.T).max() < 1e-12


def test_su2_displaced_green_is_independent_of_n_wrap_at_large_beta(orc):
    rng = np.random.default_rng(4)
    K = W.square_lattice(4, 4, t=1.0, mu=0.2)
    f = rng.choice([-2, -1, 1, 2], size=(100, 16)).astype(np.int8)     # beta = 10
    for tau in (30, 57):
        a0, b0 = orc.su2_green_displaced(K, 0.1, 4.0, 5, f, tau)
        a1, b1 = orc.su2_green_displaced(K, 0.1, 4.0, 10, f, tau)
        assert np.abs(a0 - a1).max() < 1e-10 and np.abs(b0 - b1).max() < 1e-10, tau


def test_su2_single_configuration_per_ordered_pair_equals_fock_trace(orc):
    """One four-valued field configuration of the SU(2) decoupling, every ordered
    pair its own class, on a 3-site chain without reflection symmetry: the Wick
    values of orc_su2_correlations on the configuration's complex G(0) equal
    Tr[O U_C] / Tr[U_C], U_C = U_L ... U_1, U_tau = exp(-dtau H_T)
    exp(i g sum_x eta(l_x,tau) n_x) on both colors (the constant -i g sum eta of
    (n_x - 1) cancels in the ratio).  This fixes the order of the two sites in the
    Green-function estimator per configuration, which the averages over all fields
    cannot."""
    from scipy.linalg import expm
    N, U, dtau, L = 3, 4.0, 0.25, 3
    K = W.chain_lattice(N, t=1.0, mu=0.3)
    K[0, 0] -= 0.4
    K[1, 2] = K[2, 1] = -0.7
    g = np.sqrt(0.5 * dtau * U)
    eta = {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)}
    F = Fock(N)
    ET = expm(-dtau * F.hopping(K))
    cls = np.arange(N * N, dtype=np.int32)
    cu = [F.c[F.mode(0, x)] for x in range(N)]
    cd = [F.c[F.mode(1, x)] for x in range(N)]
    for seed in (3, 4):
        f = np.random.default_rng(seed).choice([-2, -1, 1, 2], size=(L, N)).astype(np.int8)
        Uc = np.eye(F.dim, dtype=complex)
        for t in range(L):
            V = sum(1j * g * eta[int(f[t, x])] * (F.n(0, x) + F.n(1, x)) for x in range(N))
            Uc = ET @ expm(V) @ Uc
        Z = np.trace(Uc)
        G = orc.su2_plain(K, dtau, U, f)[0]
        got = orc.su2_correlations(G, cls, N * N)
        for x in range(N):
            for y in range(N):
                szx, szy = 0.5 * (F.n(0, x) - F.n(1, x)), 0.5 * (F.n(0, y) - F.n(1, y))
                nx, ny = F.n(0, x) + F.n(1, x), F.n(0, y) + F.n(1, y)
                ops = (szx @ szy, nx @ ny, cu[x].T @ cd[x] @ cd[y].T @ cu[y], cu[x].T @ cu[y] + cd[x].T @ cd[y])
                want = np.array([np.trace(O @ Uc) / Z for O in ops])
                assert np.abs(got[x * N + y] - want).max() < 1e-10, (seed, x, y, got[x * N + y], want)
        # with one G for both colors the two-body terms are symmetric in x, y, but
        # sum_s <c+_x c_y> = 2 (delta - G_yx) is not: the pin fixes the order there
        assert abs(got[0 * N + 2, 3] - got[2 * N + 0, 3]) > 1e-3


@pytest.mark.parametrize("mu", [0.0, 0.5])
def test_su2_sweep_equals_brute_force_metropolis_on_full_weights(orc, mu):
    """The SU(2) chain replayed proposal by proposal with the Metropolis rule on
    W = |Re e^{-S}| (Sec. 2.2), every weight recomputed from scratch as
    prod gamma(l)/4 e^{-i g sum eta} det(1 + B)^2 (plain product): the oracle's
    sweep (ratios from the Green function at the vertex, carried phase) makes the
    same decisions, so the fields and the carried phase agree after every sweep."""
    K, U, dtau, L = W.chain_lattice(3, t=1.0, mu=mu), 4.0, 0.25, 4
    K[0, 0] -= 0.3
    N = 3
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}

    def full_weight(f):
        _, la, ar, ph, _, _ = orc.su2_plain(K, dtau, U, f)
        return np.prod([gam[int(l)] / 4.0 for l in f.ravel()]) * np.exp(1j * ph) * np.exp(2.0 * (la + 1j * ar))

    def uniforms(seed, chain, sweep, tau, direction, vertex):
        o = orc.philox4x32_10([sweep & 0xFFFFFFFF, 2 * tau + direction, vertex, sweep >> 32],
                              [seed & 0xFFFFFFFF, ((seed >> 32) ^ chain) & 0xFFFFFFFF])
        return orc.u01(int(o[0]), int(o[1])), orc.u01(int(o[2]), int(o[3]))

    seed = 2468
    for chain in range(3):
        f = orc.init_fields(2, L, N, seed, chain).reshape(L, N)
        ch = orc.Su2Chain(K, dtau, U, f, seed=seed, chain=chain)
        f = f.copy()
        w = full_weight(f)
        for sweep in range(3):
            for direction in (0, 1):
                for step in range(L):
                    tau = L - step if direction else step + 1
                    for q in range(N):
                        x = N - 1 - q if direction else q
                        u1, u2 = uniforms(seed, chain, sweep, tau, direction, x)
                        others = [l for l in (-2, -1, 1, 2) if l != f[tau - 1, x]]
                        f1 = f.copy()
                        f1[tau - 1, x] = others[min(int(np.floor(3.0 * u1)), 2)]
                        w1 = full_weight(f1)
                        if u2 < min(1.0, abs(w1.real) / abs(w.real)):
                            f, w = f1, w1
            ch.sweep()
            assert np.array_equal(ch.fields.reshape(L, N), f), (chain, sweep)
            P = complex(ch.phase[0], ch.phase[1])
            assert abs(P / abs(P) - w / abs(w)) < 1e-9, (chain, sweep, P, w)
