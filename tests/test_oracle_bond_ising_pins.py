"""Pins of the oracle's Hubbard model coupled to a transverse Ising field on
bonds (Sec. 6: the hopping on bond b gains xi Z_b, the bond spins carry a
transverse field h and a coupling J between neighbouring bonds;
orc_hubbard_ising_plain on fixed fields, orc_ising_bond_logweight for the
bond spins' own weight).

* Exact enumeration of all four-valued HS fields and bond spins of small
  clusters, each weighted by prod gamma/4, the HS phase, det(1 + B)^2 and the
  bond spins' weight, equals the trace of the Trotter product on Fock (x) Ising
  space: the partition function and <H_T>.  Three open sites (two bonds that
  share a site) with U > 0 over two slices and at U = 0 over four slices, and
  two sites with U > 0 over three slices, at and away from half filling.
* The bond spins' weight alone: one bond, J = 0, sums to the transverse-field
  Ising chain's closed form 2 cosh(L dtau h); two bonds with J reproduce the
  transfer-matrix trace.
* xi = 0 decouples: the fermion part equals the SU(2) Hubbard oracle.
* At half filling on the bipartite chain every weight is real and positive.
* The Green function seen by a factor of the propagator (orc_hubbard_ising_green_at)
  gives the weight ratio of a bond flip as a 2 x 2 determinant and of an HS
  change as a 1 x 1 one, equal to det(1 + B') / det(1 + B) of the plain product;
  the rank-2 (Woodbury) update of it (orc_bond_rank2_update) equals the Green
  function recomputed on the flipped configuration; at the last factor it is the
  plain product's G.
* The complex UDV chain of the bond model (orc_hubbard_ising_green_udv) equals
  the plain product at beta = 1.5 (G at every slice boundary, log|det|, arg
  det), is independent of n_wrap at beta = 10 and gives the same log|det| and
  arg det at every tau.
* The Markov chain over HS fields and bond spins (orc_hubbard_ising_sweep),
  reweighted by sign e^{-S} / Re e^{-S}, reproduces <H_T> and <(sum_b Z_b)^2>
  of the Trotter product within 4 sigma over 24 independent chains, at and away
  from half filling.
"""
import itertools
import math

import numpy as np
import pytest

from paper_1704_00131_gb300 import workloads as W

from .fock_ed import Fock, hubbard_ising_trotter


def enumerate_model(orc, K, U, dtau, L, bonds, xi, h, J, pairs, hs_values):
    N, nb = K.shape[0], len(bonds)
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}
    Z, KZ, weights = 0.0, 0.0, []
    for zs in itertools.product((-1, 1), repeat=nb * L):
        z = np.array(zs, dtype=np.int8).reshape(L, nb)
        wz = math.exp(orc.ising_bond_logweight(z, dtau, h, J, pairs))
        for ls in itertools.product(hs_values, repeat=N * L):
            f = np.array(ls, dtype=np.int8).reshape(L, N)
            _, la, ar, ph, kin = orc.hubbard_ising_plain(K, bonds, xi, dtau, U, f, z)
            w = wz * np.prod([gam[l] / 4.0 for l in ls]) * np.exp(1j * ph) * np.exp(2.0 * (la + 1j * ar))
            weights.append(w)
            Z += w
            KZ += w * kin
    return Z, KZ / Z, np.array(weights)


def reference(orc, K, U, dtau, L, bonds, xi, h, J, pairs):
    eta = {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)}
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}
    return hubbard_ising_trotter(Fock(K.shape[0]), K, U, dtau, L, eta, gam, bonds, xi, h, J, pairs)


def test_enumeration_equals_trotter_trace_two_bonds_interacting(orc):
    # two bonds through site 1 with U > 0 on a chain without reflection symmetry:
    # the order of the bond factors within a slice, relative to the HS factor and
    # exp(-dtau T), changes Z and <H_T> (at U = 0, or on the symmetric chain, it
    # does not: transposing the product or reflecting the chain reverses it)
    K, U, dtau, L = W.chain_lattice(3, t=1.0, mu=0.25), 2.5, 0.3, 2
    K[0, 0] -= 0.5
    K[1, 2] = K[2, 1] = -0.8
    bonds, pairs = [(0, 1), (1, 2)], [(0, 1)]
    xi, h, J = 0.8, 0.7, 0.5
    Z, kin, _ = enumerate_model(orc, K, U, dtau, L, bonds, xi, h, J, pairs, (-2, -1, 1, 2))
    Zf, kf = reference(orc, K, U, dtau, L, bonds, xi, h, J, pairs)
    assert Z == pytest.approx(Zf, rel=1e-11)
    assert kin == pytest.approx(kf, rel=1e-10, abs=1e-12)


def test_enumeration_equals_trotter_trace_two_bonds_free_fermions(orc):
    # at U = 0 the HS field drops out (sum gamma / 4 = 1): one field value with weight 4^(N L)
    K, dtau, L = W.chain_lattice(3, t=1.0, mu=0.3), 0.2, 4
    bonds, pairs = [(0, 1), (1, 2)], [(0, 1)]
    xi, h, J = 0.7, 0.9, 0.4
    Z, kin, _ = enumerate_model(orc, K, 0.0, dtau, L, bonds, xi, h, J, pairs, (1,))
    g1 = orc.field_gamma(2, 1) / 4.0
    Z /= g1 ** (3 * L)
    Zf, kf = reference(orc, K, 0.0, dtau, L, bonds, xi, h, J, pairs)
    assert Z == pytest.approx(Zf, rel=1e-11)
    assert kin == pytest.approx(kf, rel=1e-10, abs=1e-12)


@pytest.mark.parametrize("mu", [0.0, 0.35])
def test_enumeration_equals_trotter_trace_interacting(orc, mu):
    K, U, dtau, L = W.chain_lattice(2, t=1.0, mu=mu), 3.0, 0.25, 3
    bonds, pairs = [(0, 1)], []
    xi, h, J = 0.6, 0.8, 0.0
    Z, kin, w = enumerate_model(orc, K, U, dtau, L, bonds, xi, h, J, pairs, (-2, -1, 1, 2))
    Zf, kf = reference(orc, K, U, dtau, L, bonds, xi, h, J, pairs)
    assert Z == pytest.approx(Zf, rel=1e-11)
    assert abs(Z.imag) < 1e-11 * abs(Z)
    assert kin == pytest.approx(kf, rel=1e-10, abs=1e-12)
    if mu == 0.0:
        assert np.abs(w.imag).max() < 1e-12 * np.abs(w).max() and (w.real > 0).all()
    else:
        assert np.abs(w.imag).max() > 1e-6 * np.abs(w).max()


def test_bond_spin_weight_closed_forms(orc):
    dtau, h, L = 0.15, 1.3, 5
    tot = sum(math.exp(orc.ising_bond_logweight(np.array(z, dtype=np.int8).reshape(L, 1), dtau, h, 0.0, []))
              for z in itertools.product((-1, 1), repeat=L))
    assert tot == pytest.approx(2.0 * math.cosh(L * dtau * h), rel=1e-13)
    # two coupled bonds: trace of the transfer matrix exp(dtau J Z Z) exp(dtau h (X_0 + X_1))
    J, L = 0.7, 3
    tot = sum(math.exp(orc.ising_bond_logweight(np.array(z, dtype=np.int8).reshape(L, 2), dtau, h, J, [(0, 1)]))
              for z in itertools.product((-1, 1), repeat=2 * L))
    X = np.array([[math.cosh(dtau * h), math.sinh(dtau * h)], [math.sinh(dtau * h), math.cosh(dtau * h)]])
    D = np.diag([math.exp(dtau * J), math.exp(-dtau * J), math.exp(-dtau * J), math.exp(dtau * J)])
    T = D @ np.kron(X, X)
    assert tot == pytest.approx(np.trace(np.linalg.matrix_power(T, L)), rel=1e-13)


def test_zero_coupling_reduces_to_su2_hubbard(orc):
    K, U, dtau, L = W.square_lattice(2, 2, t=1.0, mu=0.2), 4.0, 0.1, 6
    rng = np.random.default_rng(5)
    f = rng.choice(np.array([-2, -1, 1, 2], dtype=np.int8), size=(L, 4))
    z = rng.choice(np.array([-1, 1], dtype=np.int8), size=(L, 4))
    G, la, ar, ph, kin = orc.hubbard_ising_plain(K, [(0, 1), (2, 3), (0, 2), (1, 3)], 0.0, dtau, U, f, z)
    G2, la2, ar2, ph2, kin2, _ = orc.su2_plain(K, dtau, U, f.ravel())
    assert np.abs(G - G2).max() < 1e-13 and la == pytest.approx(la2, rel=1e-13)
    assert ar == pytest.approx(ar2, abs=1e-12) and ph == ph2 and kin == pytest.approx(kin2, rel=1e-12)


def random_config(rng, L, N, nb):
    hs = rng.choice(np.array([-2, -1, 1, 2], dtype=np.int8), size=(L, N))
    z = rng.choice(np.array([-1, 1], dtype=np.int8), size=(L, nb))
    return hs, z


def test_vertex_green_ratios_and_rank2_update(orc):
    K = W.chain_lattice(4, t=1.0, mu=0.3, periodic=True)
    K[0, 0] -= 0.4
    bonds = [(0, 1), (1, 2), (2, 3), (3, 0)]
    xi, dtau, U, L = 0.6, 0.15, 3.0, 5
    nb = len(bonds)
    rng = np.random.default_rng(11)
    hs, z = random_config(rng, L, 4, nb)
    G0, la0, ar0, _, _ = orc.hubbard_ising_plain(K, bonds, xi, dtau, U, hs, z)
    assert np.abs(orc.hubbard_ising_green_at(K, bonds, xi, dtau, U, hs, z, L, nb + 1) - G0).max() < 1e-13
    worst_r, worst_g = 0.0, 0.0
    for tau in (1, 3, L):
        for b in range(nb):
            part = nb - b                                    # bonds act in the order nb-1, ..., 0
            Gt = orc.hubbard_ising_green_at(K, bonds, xi, dtau, U, hs, z, tau, part)
            a = -dtau * xi * z[tau - 1, b]
            delta = np.array([[math.cosh(2 * a) - 1.0, -math.sinh(2 * a)], [-math.sinh(2 * a), math.cosh(2 * a) - 1.0]])
            G1, r = orc.bond_rank2_update(Gt, bonds[b][0], bonds[b][1], delta)
            z1 = z.copy()
            z1[tau - 1, b] *= -1
            _, la1, ar1, _, _ = orc.hubbard_ising_plain(K, bonds, xi, dtau, U, hs, z1)
            worst_r = max(worst_r, abs(r - np.exp((la1 - la0) + 1j * (ar1 - ar0))) / abs(r))
            G1r = orc.hubbard_ising_green_at(K, bonds, xi, dtau, U, hs, z1, tau, part)
            worst_g = max(worst_g, np.abs(G1 - G1r).max())
        # an HS change at site x: 1 x 1 ratio with the Green function after the HS factor
        Gt = orc.hubbard_ising_green_at(K, bonds, xi, dtau, U, hs, z, tau, 0)
        g = math.sqrt(0.5 * dtau * U)
        for x in range(4):
            l0 = int(hs[tau - 1, x])
            l1 = -l0
            d = np.exp(1j * g * (orc.field_coupling(2, 1.0, 2.0, l1) - orc.field_coupling(2, 1.0, 2.0, l0))) - 1.0
            hs1 = hs.copy()
            hs1[tau - 1, x] = l1
            _, la1, ar1, _, _ = orc.hubbard_ising_plain(K, bonds, xi, dtau, U, hs1, z)
            r = 1.0 + d * (1.0 - Gt[x, x])
            worst_r = max(worst_r, abs(r - np.exp((la1 - la0) + 1j * (ar1 - ar0))) / abs(r))
    assert worst_r < 1e-12 and worst_g < 1e-12, (worst_r, worst_g)


def test_rank2_update_with_a_general_delta(orc):
    """The rank-2 update against its definition for any change (1 + Delta) F of the
    factor F seen by G~ = (1 + F R)^-1, with Delta nonzero only on the block {i, j}:
    G~' = (1 + (1 + Delta) F R)^-1 and ratio = det(1 + (1 + Delta) F R) / det(1 + F R),
    here with a random complex F R and a random non-symmetric complex 2 x 2 block, so
    that a transposed or misplaced delta cannot pass."""
    rng = np.random.default_rng(12)
    N = 5
    A = 0.4 * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    G = np.linalg.inv(np.eye(N) + A)
    for i, j in ((1, 3), (4, 0)):
        d = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
        D = np.zeros((N, N), dtype=complex)
        D[np.ix_([i, j], [i, j])] = d
        A1 = (np.eye(N) + D) @ A
        G1_ref = np.linalg.inv(np.eye(N) + A1)
        r_ref = np.linalg.det(np.eye(N) + A1) / np.linalg.det(np.eye(N) + A)
        G1, r = orc.bond_rank2_update(G, i, j, d)
        assert np.abs(G1 - G1_ref).max() < 1e-12 * max(1.0, np.abs(G1_ref).max())
        assert abs(r - r_ref) < 1e-12 * abs(r_ref)


@pytest.mark.parametrize("mu", [0.0, 0.3])
def test_sampler_matches_trotter_product(orc, mu):
    from paper_1704_00131_gb300 import analysis as A
    K, U, dtau, L = W.chain_lattice(3, t=1.0, mu=mu), 2.0, 0.25, 4
    bonds, pairs = [(0, 1), (1, 2)], [(0, 1)]
    xi, h, J = 0.7, 0.8, 0.4
    _, kin_ref, m2_ref = hubbard_ising_trotter(Fock(3), K, U, dtau, L,
                                               {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)},
                                               {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)},
                                               bonds, xi, h, J, pairs, with_m2=True)
    n_chains, burn, n = 24, 30, 200
    rng = np.random.default_rng(3)
    ks, ms, ss = np.zeros(n_chains), np.zeros(n_chains), np.zeros(n_chains)
    acc_total = 0
    for c in range(n_chains):
        hs, z = random_config(rng, L, 3, 2)
        ch = orc.HubbardIsingChain(K, bonds, xi, h, J, pairs, dtau, U, hs, z, seed=1234, chain=c)
        for _ in range(burn):
            ch.sweep()
        for _ in range(n):
            k, s, m2, acc = ch.sweep()
            ks[c] += k.real
            ms[c] += m2.real
            ss[c] += s
            acc_total += acc
    assert 0.05 < acc_total / (n_chains * n * 2 * L * 5) < 0.95
    for est, ref in ((ks, kin_ref.real), (ms, m2_ref.real)):
        mean, err = A.jackknife(est / n, ss / n)
        assert abs(mean - ref) < 4.0 * err, (mean, err, ref)
        assert err < 0.05 * abs(ref)


def square_bonds(Lx, Ly):
    idx = lambda x, y: (x % Lx) + Lx * (y % Ly)
    return [(idx(x, y), idx(x + 1, y)) for y in range(Ly) for x in range(Lx)] + \
           [(idx(x, y), idx(x, y + 1)) for y in range(Ly) for x in range(Lx)]


def test_udv_chain_agrees_with_plain_product(orc):
    K = W.square_lattice(3, 3, t=1.0, mu=0.2)
    bonds = square_bonds(3, 3)
    xi, dtau, U, L = 0.4, 0.1, 4.0, 15
    rng = np.random.default_rng(21)
    hs, z = random_config(rng, L, 9, len(bonds))
    G0, la0, ar0, _, _ = orc.hubbard_ising_plain(K, bonds, xi, dtau, U, hs, z)
    for nw in (1, 4, 15):
        for tau in (0, 6, L):
            Gu, lu, au = orc.hubbard_ising_green_udv(K, bonds, xi, dtau, U, nw, hs, z, tau)
            Gp = G0 if tau in (0, L) else orc.hubbard_ising_green_at(K, bonds, xi, dtau, U, hs, z, tau, len(bonds) + 1)
            assert np.abs(Gu - Gp).max() < 1e-10, (nw, tau)
            assert lu == pytest.approx(la0, rel=1e-11)
            assert abs(np.angle(np.exp(1j * (au - ar0)))) < 1e-10


def test_udv_chain_low_temperature(orc):
    """beta = 10: chunk sizes agree on G, and log|det| and arg det do not depend on tau."""
    K = W.square_lattice(3, 3, t=1.0, mu=0.3)
    bonds = square_bonds(3, 3)
    xi, dtau, U, L = 0.5, 0.1, 4.0, 100
    rng = np.random.default_rng(8)
    hs, z = random_config(rng, L, 9, len(bonds))
    ref = orc.hubbard_ising_green_udv(K, bonds, xi, dtau, U, 10, hs, z, 40)
    for nw in (5, 4):
        G, la, ar = orc.hubbard_ising_green_udv(K, bonds, xi, dtau, U, nw, hs, z, 40)
        assert np.abs(G - ref[0]).max() < 1e-9 and la == pytest.approx(ref[1], rel=1e-11)
        assert abs(np.angle(np.exp(1j * (ar - ref[2])))) < 1e-9
    for tau in (0, 30, 55, 100):
        _, la, ar = orc.hubbard_ising_green_udv(K, bonds, xi, dtau, U, 10, hs, z, tau)
        assert la == pytest.approx(ref[1], rel=1e-11) and abs(np.angle(np.exp(1j * (ar - ref[2])))) < 1e-9


def _uniforms(orc, seed, chain, sweep, tau, direction, vertex):
    """The two uniforms of one proposal: Philox4x32-10 with counter
    (sweep_lo, 2 tau + dir, vertex, sweep_hi) and key (seed_lo, seed_hi ^ chain)."""
    ctr = [sweep & 0xFFFFFFFF, 2 * tau + direction, vertex, sweep >> 32]
    key = [seed & 0xFFFFFFFF, ((seed >> 32) ^ chain) & 0xFFFFFFFF]
    o = orc.philox4x32_10(ctr, key)
    return orc.u01(int(o[0]), int(o[1])), orc.u01(int(o[2]), int(o[3]))


@pytest.mark.parametrize("mu", [0.0, 0.6])
def test_sweep_equals_brute_force_metropolis_on_full_weights(orc, mu):
    """The chain over HS fields and bond spins, replayed proposal by proposal with
    the Metropolis rule on W = |Re e^{-S}| (Sec. 2.2), each weight recomputed from
    scratch: prod gamma(l)/4 e^{-i g sum eta} det(1 + B)^2 (plain product, both
    colors) times the bond spins' weight e^{S0}.  The oracle's sweep -- which
    takes its ratios from the Green function at the vertex and the rank-1 / rank-2
    determinant formulas, and carries the phase -- must make the same decisions:
    fields, spins and carried phase equal after every sweep.  Away from half
    filling the weights are complex, so sampling |e^{-S}| instead of |Re e^{-S}|
    changes decisions."""
    K, U, dtau, L = W.chain_lattice(3, t=1.0, mu=mu), 4.0, 0.25, 4
    K[0, 0] -= 0.3
    bonds, pairs = [(0, 1), (1, 2)], [(0, 1)]
    xi, h, J = 0.7, 0.8, 0.4
    N, nb = 3, 2
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}

    def full_weight(hs, z):
        _, la, ar, ph, _ = orc.hubbard_ising_plain(K, bonds, xi, dtau, U, hs, z)
        g = np.prod([gam[int(l)] / 4.0 for l in hs.ravel()])
        return g * np.exp(1j * ph) * np.exp(2.0 * (la + 1j * ar)) * np.exp(orc.ising_bond_logweight(z, dtau, h, J, pairs))

    seed, n_sweeps, decisions = 4321, 3, 0
    for chain in range(3):
        rng = np.random.default_rng(chain)
        hs, z = random_config(rng, L, N, nb)
        ch = orc.HubbardIsingChain(K, bonds, xi, h, J, pairs, dtau, U, hs, z, seed=seed, chain=chain)
        hs, z = hs.copy(), z.copy()
        w = full_weight(hs, z)
        for sweep in range(n_sweeps):
            for direction in (0, 1):
                for step in range(L):
                    tau = L - step if direction else step + 1
                    for q in range(N + nb):
                        v = N + nb - 1 - q if direction else q
                        hs1, z1 = hs.copy(), z.copy()
                        if v < N:
                            u1, u2 = _uniforms(orc, seed, chain, sweep, tau, direction, v)
                            others = [l for l in (-2, -1, 1, 2) if l != hs[tau - 1, v]]
                            hs1[tau - 1, v] = others[min(int(np.floor(3.0 * u1)), 2)]
                        else:
                            b = nb - 1 - (v - N)
                            u1, u2 = _uniforms(orc, seed, chain, sweep, tau, direction, N + b)
                            z1[tau - 1, b] = -z1[tau - 1, b]
                        w1 = full_weight(hs1, z1)
                        if u2 < min(1.0, abs(w1.real) / abs(w.real)):
                            hs, z, w = hs1, z1, w1
                        decisions += 1
            ch.sweep()
            assert np.array_equal(ch.hs.reshape(L, N), hs) and np.array_equal(ch.ising.reshape(L, nb), z), (chain, sweep)
            P = complex(ch.phase[0], ch.phase[1])
            assert abs(P / abs(P) - w / abs(w)) < 1e-9, (chain, sweep, P, w)
    assert decisions == 3 * n_sweeps * 2 * L * (N + nb)
