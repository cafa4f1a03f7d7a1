"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here runs on the CPU (no GPU marker).  Each one is chosen so that a
plausible mistake in the oracle (a dropped term, a wrong sign or index, a
transposed operand) fails it:

* Philox4x32-10 known-answer vectors (published with the generator);
* the discrete HS constants of Sec. 2.1 and the exact Ising decoupling;
* U = 0 closed forms: G(tau) = (1 + exp(-beta K))^-1 at every tau, log det and
  kinetic energy from the lattice dispersion;
* exact enumeration of every field configuration of 2- and 4-site clusters
  against the Fock-space trace of the Trotterised density matrix (ED);
* particle-hole symmetry at half filling on bipartite lattices;
* the UDV chain against the plain product, and n_wrap independence;
* the fast-updated, wrapped G against the freshly stabilised one, and the sign
  carried through negative ratios against the recomputed one;
* central finite differences of log|det(1 + B(beta,0))|;
* Monte Carlo estimates of the sampler against ED within 3 sigma.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm

from paper_1704_00131_gb300 import workloads as W
from tests.fock_ed import Fock

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def make_model(orc, K, U, dtau, L, nwrap, ft=1, nfl=2):
    N = K.shape[-1]
    H = K if K.ndim == 3 else np.stack([K] * nfl)
    sign = np.stack([np.ones(N), -np.ones(N)])[:nfl]
    return orc.Model(H, np.arange(N, dtype=np.int32), sign, U, dtau, L, nwrap, ft)


# --------------------------------------------------------------------------- RNG
def test_philox_known_answers(orc):
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert list(orc.philox4x32_10(w[0:4], w[4:6])) == w[6:10]
        n += 1
    assert n == 3


def test_uniform_mapping(orc):
    assert orc.u01(0, 0) == 0.0
    assert orc.u01(0x80000000, 0) == 0.5
    assert orc.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    # 53 bits: the 11 lowest bits of the low word are dropped
    assert orc.u01(0, 0x7FF) == 0.0 and orc.u01(0, 0x800) == 2.0 ** -53


def test_init_fields_distribution(orc):
    f = orc.init_fields(1, 200, 50, seed=7, chain=3)
    assert set(np.unique(f)) == {-1, 1}
    assert abs(f.mean()) < 0.05
    g = orc.init_fields(2, 200, 50, seed=7, chain=3)
    assert set(np.unique(g)) == {-2, -1, 1, 2}
    for v in (-2, -1, 1, 2):
        assert abs((g == v).mean() - 0.25) < 0.02
    assert not np.array_equal(f, orc.init_fields(1, 200, 50, seed=7, chain=4))


# ------------------------------------------------------------ HS transformations
def test_hs4_constants_match_paper_identity(orc):
    """(1/4) sum_l gamma(l) exp(a eta(l) A) = exp(a^2 A^2) + O(a^8) (Sec. 2.1, Eq. HS_squares,
    with the 1/4 normalisation of the weights; a^2 = dtau*lambda, so the error is O(dtau^4))."""
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}
    s6 = math.sqrt(6.0)
    assert gam[1] == pytest.approx(1 + s6 / 3, rel=1e-15) and gam[-2] == pytest.approx(1 - s6 / 3, rel=1e-15)
    # eta(l) from the coupling with dtau*U/2 = 1, i.e. g = 1
    eta = {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)}
    assert eta[1] == pytest.approx(math.sqrt(2 * (3 - s6)), rel=1e-15)
    assert eta[-2] == pytest.approx(-math.sqrt(2 * (3 + s6)), rel=1e-15)
    for A in (0.0, 1.0, 2.0):
        errs = []
        for a in (0.1, 0.05):
            lhs = sum(gam[l] * math.exp(a * eta[l] * A) for l in gam) / 4.0
            errs.append(abs(lhs - math.exp(a * a * A * A)))
        if A == 0.0:
            assert max(errs) < 1e-15
        else:
            # O(a^8): halving a divides the error by ~2^8
            assert errs[1] < errs[0] / 150.0


def test_ising_decoupling_is_exact(orc):
    """(1/2) e^{-dtau U/4} sum_s e^{lambda s (n_up - n_dn)} = e^{-dtau U (n_up-1/2)(n_dn-1/2)}."""
    for dtau, U in ((0.1, 4.0), (0.05, 2.0), (0.2, 6.0)):
        lam = orc.ising_lambda(dtau, U)
        assert orc.field_coupling(1, dtau, U, 1) == pytest.approx(lam, rel=1e-15)
        for nu, nd in itertools.product((0, 1), (0, 1)):
            lhs = 0.5 * math.exp(-dtau * U / 4) * sum(math.exp(lam * s * (nu - nd)) for s in (1, -1))
            rhs = math.exp(-dtau * U * (nu - 0.5) * (nd - 0.5))
            assert lhs == pytest.approx(rhs, rel=1e-14)


# ------------------------------------------------------------------ dense algebra
def test_eig_and_expm_against_library(orc):
    rng = np.random.default_rng(1)
    for n in (1, 5, 16):
        A = rng.standard_normal((n, n))
        A = A + A.T
        w, V = orc.eig_sym(A)
        assert np.allclose(np.sort(w), np.linalg.eigvalsh(A), atol=1e-12)
        assert np.allclose(V @ np.diag(w) @ V.T, A, atol=1e-12)
        assert np.allclose(orc.expm_sym(A, -0.3), expm(-0.3 * A), rtol=1e-12, atol=1e-13)


def test_logdet_against_library(orc):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((9, 9))
    ld, sg = orc.logdet(A)
    s2, l2 = np.linalg.slogdet(A)
    assert ld == pytest.approx(l2, rel=1e-13) and sg == int(s2)


# ---------------------------------------------------------------- U = 0 closed form
def square_dispersion(Lx, Ly, t, tp, mu):
    e = []
    for ny in range(Ly):
        for nx in range(Lx):
            kx, ky = 2 * np.pi * nx / Lx, 2 * np.pi * ny / Ly
            e.append(-2 * t * (np.cos(kx) + np.cos(ky)) - 4 * tp * np.cos(kx) * np.cos(ky) - mu)
    return np.sort(np.array(e))


def honeycomb_dispersion(L1, L2, t, mu):
    a1 = np.array([1.0, 0.0])
    a2 = np.array([0.5, np.sqrt(3) / 2])
    # reciprocal vectors g_i with a_i . g_j = 2 pi delta_ij
    Amat = np.stack([a1, a2])
    G = 2 * np.pi * np.linalg.inv(Amat).T
    e = []
    for n2 in range(L2):
        for n1 in range(L1):
            k = n1 / L1 * G[0] + n2 / L2 * G[1]
            f = 1 + np.exp(1j * k @ (a1 - a2)) + np.exp(-1j * k @ a2)
            e += [t * abs(f) - mu, -t * abs(f) - mu]
    return np.sort(np.array(e))


@pytest.mark.parametrize("lattice", ["square4x4", "square4x4_tp_mu", "honeycomb3x3"])
def test_free_fermion_closed_form(orc, lattice):
    if lattice == "square4x4":
        K, eps, dtau, L = W.square_lattice(4, 4), square_dispersion(4, 4, 1.0, 0.0, 0.0), 0.1, 20
    elif lattice == "square4x4_tp_mu":
        K, eps, dtau, L = (W.square_lattice(4, 4, 1.0, -0.2, -0.5), square_dispersion(4, 4, 1.0, -0.2, -0.5), 0.05, 40)
    else:
        K, eps, dtau, L = W.honeycomb_lattice(3, 3), honeycomb_dispersion(3, 3, 1.0, 0.0), 0.1, 30
    beta = dtau * L
    # the lattice builder reproduces the analytic band structure
    assert np.allclose(np.linalg.eigvalsh(K), eps, atol=1e-12)
    m = make_model(orc, K, 0.0, dtau, L, 10)
    N = K.shape[0]
    fields = W.random_fields(1, L, N, seed=3)  # irrelevant at U = 0
    w, V = np.linalg.eigh(K)
    Gexact = V @ np.diag(1.0 / (1.0 + np.exp(-beta * w))) @ V.T
    ld_exact = np.sum(np.log1p(np.exp(-beta * eps)))
    for tau in (0, 7, L):
        for fn in (orc.green_plain, orc.green_udv):
            G, ld, sg = fn(m, fields, 0, tau)
            assert np.allclose(G, Gexact, atol=1e-12), (fn.__name__, tau)
            assert ld == pytest.approx(ld_exact, rel=1e-12, abs=1e-12) and sg == 1
    kin_exact = 2 * np.sum(eps / (1.0 + np.exp(beta * eps)))
    e = orc.energy(m, np.stack([Gexact, Gexact]))
    assert e[0] == pytest.approx(kin_exact, rel=1e-12, abs=1e-12)
    n_exact = 2 * np.sum(1.0 / (1.0 + np.exp(beta * eps)))
    assert e[2] == pytest.approx(n_exact, rel=1e-12)
    # a chain at U = 0 accepts every proposal and its G never leaves the closed form
    ch = orc.Chain(m, fields, seed=5, measure=True)
    st = ch.sweep(1)
    assert st.accepted == st.proposals == 2 * L * N
    assert np.allclose(ch.green(1), Gexact, atol=1e-12)
    assert st.prec_green_max < 1e-12
    meas, ssum, nm = ch.measure()
    assert nm == 2 * L and ssum == nm
    assert meas[0] / nm == pytest.approx(kin_exact, rel=1e-11, abs=1e-11)


def test_free_fermion_logdet_gradient_closed_form(orc):
    """At U = 0, log det(1 + e^{-beta K}) has d/dK_xy = -beta (1 - G)_yx exactly."""
    K = W.square_lattice(4, 4)
    L, dtau = 10, 0.1
    m = make_model(orc, K, 0.0, dtau, L, 5)
    fields = W.random_fields(1, L, 16, seed=1)
    ld, sg, gK, gU = orc.logdet_grad(m, fields)
    w, V = np.linalg.eigh(K)
    G = V @ np.diag(1.0 / (1.0 + np.exp(-L * dtau * w))) @ V.T
    g = -L * dtau * (np.eye(16) - G).T
    gsym = g + g.T - np.diag(np.diag(g))
    for s in range(2):
        assert np.allclose(gK[s], gsym, atol=1e-11)


# ----------------------------------------------------- exact enumeration vs ED
def enumerate_ising(orc, K, U, dtau, L):
    N = K.shape[0]
    m = make_model(orc, K, U, dtau, L, L)
    pref = (0.5 * math.exp(-dtau * U / 4.0)) ** (N * L)
    Z = 0.0
    num = np.zeros(4)
    for bits in itertools.product((-1, 1), repeat=N * L):
        f = np.array(bits, dtype=np.int8).reshape(L, N)
        G0, ld0, s0 = orc.green_plain(m, f, 0, 0)
        G1, ld1, s1 = orc.green_plain(m, f, 1, 0)
        w = pref * s0 * s1 * math.exp(ld0 + ld1)
        Z += w
        num += w * orc.energy(m, np.stack([G0, G1]))
    return Z, num / Z


@pytest.mark.parametrize("cluster", ["dimer", "plaquette"])
def test_enumeration_equals_fock_trace_ising(orc, cluster):
    if cluster == "dimer":
        K, U, dtau, L = W.chain_lattice(2, t=1.0, mu=0.3), 3.0, 0.25, 4
    else:
        K, U, dtau, L = W.square_lattice(2, 2, t=1.0), 4.0, 0.3, 4
    Z, e = enumerate_ising(orc, K, U, dtau, L)
    F = Fock(K.shape[0])
    rho = F.trotter_ising(K, U, dtau, L)
    Zed = np.trace(rho)
    assert Z == pytest.approx(Zed, rel=1e-11)
    HT = F.hopping(K)
    Hn = F.hubbard_nn(U)
    # estimators evaluated at the boundary tau = 0 of the trace
    assert e[0] == pytest.approx(np.trace(HT @ rho) / Zed, rel=1e-10, abs=1e-12)
    assert e[1] == pytest.approx(np.trace(Hn @ rho) / Zed, rel=1e-10, abs=1e-12)
    Nop = sum(F.n(s, i) for s in range(2) for i in range(K.shape[0]))
    assert e[2] == pytest.approx(np.trace(Nop @ rho) / Zed, rel=1e-10)


def test_enumeration_equals_fock_trace_hs4(orc):
    K, U, dtau, L = W.chain_lattice(2, t=1.0, mu=-0.2), 4.0, 0.2, 4
    N = 2
    m = make_model(orc, K, U, dtau, L, 2, ft=2)
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}
    eta = {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)}
    Z = 0.0
    for ls in itertools.product((-2, -1, 1, 2), repeat=N * L):
        f = np.array(ls, dtype=np.int8).reshape(L, N)
        _, ld0, s0 = orc.green_plain(m, f, 0, 0)
        _, ld1, s1 = orc.green_plain(m, f, 1, 0)
        w = np.prod([gam[l] / 4.0 for l in ls]) * s0 * s1 * math.exp(ld0 + ld1)
        Z += w
    F = Fock(N)
    Zed = np.trace(F.trotter_hs4(K, U, dtau, L, eta, gam))
    assert Z == pytest.approx(Zed, rel=1e-11)


# ------------------------------------------------------------------ symmetries
@pytest.mark.parametrize("lat", ["square", "honeycomb"])
def test_particle_hole_symmetry(orc, lat):
    if lat == "square":
        K, D = W.square_lattice(4, 4), W.sublattice_signs_square(4, 4)
    else:
        K, D = W.honeycomb_lattice(2, 3), W.sublattice_signs_honeycomb(2, 3)
    N = K.shape[0]
    L, dtau, U = 20, 0.1, 4.0
    m = make_model(orc, K, U, dtau, L, 10)
    f = W.random_fields(1, L, N, seed=11)
    lam = orc.ising_lambda(dtau, U)
    for tau in (0, 10, 13):
        Gu, ldu, su = orc.green_udv(m, f, 0, tau)
        Gd, ldd, sd = orc.green_udv(m, f, 1, tau)
        assert np.allclose(Gd, np.diag(D) @ (np.eye(N) - Gu.T) @ np.diag(D), atol=1e-12)
        assert ldd == pytest.approx(ldu - lam * f.sum(), rel=1e-12, abs=1e-10)
        assert su == sd == 1


def test_udv_agrees_with_plain_product(orc):
    K = W.square_lattice(4, 4)
    m = make_model(orc, K, 4.0, 0.1, 20, 10)
    f = W.random_fields(1, 20, 16, seed=4)
    for tau in (0, 3, 10, 17, 20):
        for s in (0, 1):
            Gp, lp, sp = orc.green_plain(m, f, s, tau)
            Gu, lu, su = orc.green_udv(m, f, s, tau)
            # the plain inverse carries eps * cond(1 + B(beta,0)) (Sec. 2.3): ~1e4 here
            assert np.abs(Gp - Gu).max() < 5e-11
            assert lu == pytest.approx(lp, rel=1e-12) and su == sp


def test_udv_sign_per_flavor_odd_lattice(orc):
    """Per flavor, the sign and log|det| of the UDV chain equal numpy's slogdet of
    1 + B(tau,0)B(beta,tau) built from plain numpy products, on an odd lattice
    (3x3 torus away from half filling) where single-flavor determinants change
    sign and an odd number of reflections enters each orthogonal factor."""
    K = W.square_lattice(3, 3, t=1.0, mu=-0.5)
    N, U, dtau, L = 9, 6.0, 0.25, 16
    m = make_model(orc, K, U, dtau, L, 4)
    lam = np.arccosh(np.exp(0.5 * dtau * U))
    E = expm(-dtau * K)
    seen = set()
    for seed in range(6):
        f = W.random_fields(1, L, N, seed=40 + seed)
        for s, sig in ((0, 1.0), (1, -1.0)):
            Bs = [E @ np.diag(np.exp(sig * lam * f[t].astype(float))) for t in range(L)]
            for tau in (0, 6, L):
                P = np.eye(N)
                for t in list(range(tau, L)) + list(range(tau)):   # B(tau,0) B(beta,tau), cyclically
                    P = Bs[t] @ P
                sg_np, ld_np = np.linalg.slogdet(np.eye(N) + P)
                # the plain product's determinant carries eps * cond(1 + B) (Sec. 2.3)
                tol = 1e-11 * abs(ld_np) + 100 * np.finfo(float).eps * np.linalg.cond(np.eye(N) + P)
                _, lu, su = orc.green_udv(m, f, s, tau)
                assert su == int(sg_np) and abs(lu - ld_np) < tol, (seed, s, tau, lu - ld_np, tol)
                seen.add(su)
    assert seen == {-1, 1}


def test_udv_independent_of_nwrap_at_low_temperature(orc):
    """beta = 10, U = 4: the plain product is hopeless, chunk sizes must agree."""
    K = W.square_lattice(4, 4)
    L = 100
    f = W.random_fields(1, L, 16, seed=9)
    ref = None
    for nw in (10, 5, 2):
        m = make_model(orc, K, 4.0, 0.1, L, nw)
        G, ld, sg = orc.green_udv(m, f, 0, 40)
        if ref is None:
            ref = (G, ld)
        else:
            assert np.abs(G - ref[0]).max() < 1e-9
            assert ld == pytest.approx(ref[1], rel=1e-11)
    # cyclicity: log det(1 + B(tau,0)B(beta,tau)) does not depend on tau
    m = make_model(orc, K, 4.0, 0.1, L, 10)
    lds = [orc.green_udv(m, f, 0, t)[1] for t in (0, 30, 55, 100)]
    assert max(lds) - min(lds) < 1e-9 * abs(lds[0])


# -------------------------------------------------------- fast updates vs fresh G
@pytest.mark.parametrize("ft", [1, 2])
def test_wrapped_sherman_morrison_matches_fresh(orc, ft):
    """With n_wrap = L the only stabilisations are at tau = L (up) and 0 (down): the
    monitor then compares G after L slices of Sherman-Morrison updates and wraps with
    the exact G on the updated fields.  Round-off grows exponentially with the number
    of unstabilised slices (Sec. 2.3), so a weak coupling keeps it measurable."""
    K = W.square_lattice(4, 4)
    m = make_model(orc, K, 2.0, 0.1, 10, 10, ft=ft)
    ch = orc.Chain(m, None, seed=123, chain=1)
    st = ch.sweep(3)
    assert 0 < st.accepted < st.proposals
    assert st.prec_green_max < 1e-10
    f, nsw, sign = ch.fields()
    assert nsw == 3
    for s in (0, 1):
        Gp, _, _ = orc.green_plain(m, f, s, 0)
        assert np.abs(ch.green(s) - Gp).max() < 1e-12


def test_trajectory_independent_of_stabilisation_interval(orc):
    """Accept/reject decisions depend on G only through the ratios, which must not change
    (beyond round-off) with the stabilisation interval: same fields for n_wrap = 1..10."""
    K = W.square_lattice(4, 4)
    ref = None
    for nw in (1, 2, 5, 10):
        m = make_model(orc, K, 4.0, 0.1, 20, nw)
        ch = orc.Chain(m, None, seed=99, chain=2)
        st = ch.sweep(3)
        f, _, _ = ch.fields()
        if ref is None:
            ref = (f, st.accepted)
        else:
            assert np.array_equal(f, ref[0]) and st.accepted == ref[1]


def test_precision_monitor_low_temperature(orc):
    """4x4, U/t = 4, beta t = 10 (the paper's precision example size): the wrapped and
    the fresh G agree to well below the recommended 1e-8 mean."""
    K = W.square_lattice(4, 4)
    m = make_model(orc, K, 4.0, 0.1, 100, 10)
    ch = orc.Chain(m, None, seed=1, chain=0)
    st = ch.sweep(2)
    assert st.prec_green_mean < 1e-8
    assert st.prec_green_max < 1e-5
    assert st.prec_phase_max == 0.0 and st.mean_sign == 1.0


def test_sign_tracked_through_negative_ratios(orc):
    """Away from half filling on the frustrated 3x3 torus the spin-z decoupling has
    negative weights: the sign carried through the updates (flipped on every
    accepted negative ratio) must equal the sign of det(1 + B_up) det(1 + B_dn)
    recomputed at every stabilisation (the phase monitor of Sec. 2.3 stays 0) and
    at the end of the sweeps, while the chain visits both signs."""
    K = W.square_lattice(3, 3, t=1.0, mu=-0.5)
    m = make_model(orc, K, 6.0, 0.125, 32, 4)
    ch = orc.Chain(m, W.random_fields(1, 32, 9, seed=1).reshape(32, 9), seed=5, chain=0)
    st = ch.sweep(20)
    assert st.mean_sign < 0.99
    assert st.prec_phase_max == 0.0
    f, _, sign = ch.fields()
    want = orc.green_udv(m, f, 0, 0)[2] * orc.green_udv(m, f, 1, 0)[2]
    assert sign == want


# ---------------------------------------------------------------- derivatives
def test_logdet_gradient_finite_differences(orc):
    K = W.square_lattice(3, 2, t=1.0, tp=0.0, mu=0.2)
    N = K.shape[0]
    L, dtau, U = 8, 0.1, 3.0
    f = W.random_fields(1, L, N, seed=21)
    m = make_model(orc, K, U, dtau, L, 4)
    ld, sg, gK, gU = orc.logdet_grad(m, f)
    h = 1e-5

    def ld_of(Kp, Up):
        mm = make_model(orc, Kp, Up, dtau, L, 4)
        return np.array([orc.green_udv(mm, f, s, 0)[1] for s in (0, 1)])

    assert np.allclose(ld, ld_of(K, U), rtol=1e-12)
    for (x, y) in ((0, 1), (2, 2), (1, 4), (0, 3)):
        Kp = K.copy(); Km = K.copy()
        Kp[x, y] += h; Km[x, y] -= h
        if x != y:
            Kp[y, x] += h; Km[y, x] -= h
        fd = (ld_of(Kp, U) - ld_of(Km, U)) / (2 * h)
        assert np.allclose(gK[:, x, y], fd, rtol=1e-6, atol=1e-8), (x, y)
    fdU = (ld_of(K, U + h) - ld_of(K, U - h)) / (2 * h)
    assert np.allclose(gU, fdU, rtol=1e-6, atol=1e-8)


# ----------------------------------------------------------- sampler statistics
def jackknife(x):
    x = np.asarray(x)
    n = len(x)
    loo = (x.sum() - x) / (n - 1)
    mean = loo.mean()
    err = math.sqrt((n - 1) / n * np.sum((loo - mean) ** 2))
    return mean, err


@pytest.mark.parametrize("ft", [1, 2])
def test_sampler_reproduces_exact_energies(orc, ft):
    """Monte Carlo estimates on the 2x2 Hubbard plaquette agree with ED within 3 sigma."""
    K = W.square_lattice(2, 2, t=1.0)
    U, dtau, L = 4.0, 0.125, 8
    m = make_model(orc, K, U, dtau, L, 4, ft=ft)
    F = Fock(4)
    if ft == 1:
        rho = F.trotter_ising(K, U, dtau, L)
    else:
        gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}
        eta = {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)}
        rho = F.trotter_hs4(K, U, dtau, L, eta, gam)
    Z = np.trace(rho)
    kin_ed = np.trace(F.hopping(K) @ rho) / Z
    pot_ed = np.trace(F.hubbard_nn(U) @ rho) / Z
    bins_k, bins_p = [], []
    ch = orc.Chain(m, None, seed=77, chain=0, measure=True, meas_first=0, meas_last=L)
    ch.sweep(20)  # warm-up (measured too; discarded through the differences below)
    prev, _, prev_n = ch.measure()
    for b in range(40):
        ch.sweep(50)
        cur, _, cur_n = ch.measure()
        d = (cur - prev) / (cur_n - prev_n)
        bins_k.append(d[0])
        bins_p.append(d[1])
        prev, prev_n = cur, cur_n
    mk, ek = jackknife(bins_k)
    mp, ep = jackknife(bins_p)
    assert abs(mk - kin_ed) < 3 * ek + 1e-12, (mk, ek, kin_ed)
    assert abs(mp - pot_ed) < 3 * ep + 1e-12, (mp, ep, pot_ed)


def test_sampler_with_negative_weights_matches_exact_energies(orc):
    """Away from half filling on a frustrated ring (a triangle, mu = 0.8, U = 8,
    beta = 5) some configurations have negative weight: the chain samples |w|,
    and the estimators are the sign-reweighted <O s> / <s> (Sec. 2.2).  Kin and
    Pot from 32 chains agree with ED of the Trotterised density matrix within
    4 sigma, and the mean sign is well below 1, so an estimator that dropped the
    sign would be off by (1 - <s>) / <s> of the energy scale."""
    from paper_1704_00131_gb300 import analysis as A
    N, mu, U, dtau, L = 3, 0.8, 8.0, 0.125, 40
    K = W.chain_lattice(N, t=1.0, mu=mu, periodic=True)
    m = make_model(orc, K, U, dtau, L, 4)
    F = Fock(N)
    rho = F.trotter_ising(K, U, dtau, L)
    Z = np.trace(rho)
    kin_ed = np.trace(F.hopping(K) @ rho) / Z
    pot_ed = np.trace(F.hubbard_nn(U) @ rho) / Z
    nch, burn, n = 32, 30, 300
    os_, ss = np.zeros((nch, 4)), np.zeros(nch)
    for c in range(nch):
        ch = orc.Chain(m, None, seed=7, chain=c, measure=True, meas_first=0, meas_last=0)
        ch.sweep(burn)
        e0, s0, n0 = ch.measure()
        ch.sweep(n)
        e1, s1, n1 = ch.measure()
        os_[c] = (e1 - e0) / (n1 - n0)
        ss[c] = (s1 - s0) / (n1 - n0)
    mean, err = A.jackknife(os_, ss)
    assert ss.mean() < 0.8
    assert abs(mean[0] - kin_ed) < 4 * err[0], (mean[0], err[0], kin_ed)
    assert abs(mean[1] - pot_ed) < 4 * err[1], (mean[1], err[1], pot_ed)


# ----------------------------------------------------------- energy adjoint
def test_displaced_green_against_plain_products(orc):
    """G(tau,0) = B(tau,0) G(0) and G(0,tau) = -(1 - G(0)) B(tau,0)^-1 by plain products
    at small beta, against the UDV-chain formulas."""
    K = W.square_lattice(2, 3, 1.0, 0.0, 0.2)
    N, L, dtau, U = 6, 8, 0.1, 3.0
    m = make_model(orc, K, U, dtau, L, 4)
    f = W.random_fields(1, L, N, seed=31)
    E = expm(-dtau * K)
    lam = orc.ising_lambda(dtau, U)
    for s, sig in ((0, 1.0), (1, -1.0)):
        G0, _, _ = orc.green_plain(m, f, s, 0)
        for tau in (0, 3, 4, 8):
            B = np.eye(N)
            for t in range(1, tau + 1):
                B = E @ np.diag(np.exp(sig * lam * f[t - 1])) @ B
            Gt0, G0t = orc.green_displaced(m, f, s, tau)
            assert np.allclose(Gt0, B @ G0, atol=1e-12)
            assert np.allclose(G0t, -(np.eye(N) - G0) @ np.linalg.inv(B), atol=1e-12)


def test_energy_gradient_finite_differences(orc):
    K = W.square_lattice(3, 2, t=1.0, tp=0.0, mu=0.2)
    N = K.shape[0]
    L, dtau, U = 8, 0.1, 3.0
    for ft in (1, 2):
        f = W.random_fields(ft, L, N, seed=41 + ft)
        m = make_model(orc, K, U, dtau, L, 4, ft=ft)
        e, gK, gU = orc.energy_grad(m, f)
        h = 1e-5

        def ener(Kp, Up):
            mm = make_model(orc, Kp, Up, dtau, L, 4, ft=ft)
            G = np.stack([orc.green_udv(mm, f, s, 0)[0] for s in (0, 1)])
            return orc.energy(mm, G)[3]

        assert e[3] == pytest.approx(ener(K, U), rel=1e-12)
        for (x, y) in ((0, 1), (2, 2), (1, 4), (0, 3)):
            Kp = K.copy(); Km = K.copy()
            Kp[x, y] += h; Km[x, y] -= h
            if x != y:
                Kp[y, x] += h; Km[y, x] -= h
            fd = (ener(Kp, U) - ener(Km, U)) / (2 * h)
            # one K shared by both flavors: the total derivative is the sum over flavors
            assert gK[:, x, y].sum() == pytest.approx(fd, rel=1e-6, abs=1e-8), (ft, x, y)
        fdU = (ener(K, U + h) - ener(K, U - h)) / (2 * h)
        assert gU == pytest.approx(fdU, rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("ft", [1, 2])
def test_sweep_equals_brute_force_metropolis_on_full_weights(orc, ft):
    """The spin-z chain replayed proposal by proposal with the Metropolis rule on
    |w| (Sec. 2.2), each weight recomputed from scratch as prod_s det(1 + B_s)
    through the stabilised chain (times prod gamma(l) for the four-valued
    field; beta = 4 is beyond the plain product's reach at U = 8): the
    oracle's chain -- ratios from the wrapped Green function, Sherman-Morrison
    updates, stabilisations -- makes the same decisions and carries the same sign,
    on a frustrated triangle away from half filling where weights go negative."""
    N, mu, U, dtau, L = 3, 0.8, 8.0, 0.125, 32
    K = W.chain_lattice(N, t=1.0, mu=mu, periodic=True)
    m = make_model(orc, K, U, dtau, L, 4, ft=ft)

    def log_weight(f):
        lds = [orc.green_udv(m, f, s, 0)[1:] for s in (0, 1)]
        lg = sum(math.log(orc.field_gamma(ft, int(l))) for l in f.ravel())
        return sum(ld for ld, _ in lds) + lg, lds[0][1] * lds[1][1]

    def uniforms(seed, chain, sweep, tau, direction, vertex):
        o = orc.philox4x32_10([sweep & 0xFFFFFFFF, 2 * tau + direction, vertex, sweep >> 32],
                              [seed & 0xFFFFFFFF, ((seed >> 32) ^ chain) & 0xFFFFFFFF])
        return orc.u01(int(o[0]), int(o[1])), orc.u01(int(o[2]), int(o[3]))

    seed, negative = 97, 0
    for chain in range(4):
        f = orc.init_fields(ft, L, N, seed, chain).reshape(L, N)
        ch = orc.Chain(m, f, seed=seed, chain=chain)
        f = f.copy()
        lw, sg = log_weight(f)
        for sweep in range(3):
            for direction in (0, 1):
                for step in range(L):
                    tau = L - step if direction else step + 1
                    for q in range(N):
                        k = N - 1 - q if direction else q
                        u1, u2 = uniforms(seed, chain, sweep, tau, direction, k)
                        f1 = f.copy()
                        if ft == 1:
                            f1[tau - 1, k] = -f[tau - 1, k]
                        else:
                            others = [l for l in (-2, -1, 1, 2) if l != f[tau - 1, k]]
                            f1[tau - 1, k] = others[min(int(math.floor(3.0 * u1)), 2)]
                        lw1, sg1 = log_weight(f1)
                        if u2 < min(1.0, math.exp(lw1 - lw)):
                            f, lw, sg = f1, lw1, sg1
                            negative += sg < 0
            ch.sweep(1)
            fo, _, so = ch.fields()
            assert np.array_equal(fo, f), (chain, sweep)
            assert so == sg, (chain, sweep, so, sg)
    assert negative > 0                                  # the sign was exercised
