"""Pins of the oracle's equal-time correlation functions (orc_correlations).

* Exact enumeration of all Ising fields of small clusters, each configuration
  weighted by det(1 + B_up) det(1 + B_dn) and measured on its G(0), equals the
  Fock-space trace Tr[O rho] / Tr[rho] of the Trotterised density matrix for
  O = S^z_x S^z_y, n_x n_y, S^+_x S^-_y and sum_s c^+_xs c_ys, summed over each
  pair class.
* The same averages obey the spin-rotation symmetry of the Hubbard model:
  <S^z_x S^z_y> = (<S^+_x S^-_y> + <S^-_x S^+_y>) / 4 for x != y (per
  configuration they do not).
* Translation classes of the square lattice partition all pairs.
"""
import itertools
import math

import numpy as np
import pytest

from paper_1704_00131_gb300 import workloads as W

from .fock_ed import Fock, equal_time_correlations


def make_model(orc, K, U, dtau, L, nwrap):
    N = K.shape[-1]
    sign = np.stack([np.ones(N), -np.ones(N)])
    return orc.Model(np.stack([K, K]), np.arange(N, dtype=np.int32), sign, U, dtau, L, nwrap, 1)


@pytest.mark.parametrize("cluster", ["dimer", "plaquette"])
def test_correlations_enumeration_equals_fock_trace(orc, cluster):
    if cluster == "dimer":
        K, U, dtau, L = W.chain_lattice(2, t=1.0, mu=0.3), 3.0, 0.25, 4
        N = 2
        cls = np.array([0, 1, 1, 0], dtype=np.int32)          # on-site, neighbour
        n_class = 2
    else:
        K, U, dtau, L = W.square_lattice(2, 2, t=1.0), 4.0, 0.3, 3
        N = 4
        cls, n_class, _ = W.translation_classes_square(2, 2)
    m = make_model(orc, K, U, dtau, L, L)
    Z = 0.0
    acc = np.zeros((n_class, 4))
    for bits in itertools.product((-1, 1), repeat=N * L):
        f = np.array(bits, dtype=np.int8).reshape(L, N)
        G0, ld0, s0 = orc.green_udv(m, f, 0, 0)
        G1, ld1, s1 = orc.green_udv(m, f, 1, 0)
        w = s0 * s1 * math.exp(ld0 + ld1)
        Z += w
        acc += w * orc.correlations(np.stack([G0, G1]), cls, n_class)
    ref = equal_time_correlations(Fock(N), K, U, dtau, L, cls, n_class)
    assert acc / Z == pytest.approx(ref, rel=1e-10, abs=1e-12)


def test_spin_rotation_symmetry_of_the_average(orc):
    K, U, dtau, L = W.chain_lattice(3, t=1.0, mu=-0.1, periodic=False), 4.0, 0.25, 3
    N = 3
    cls = np.arange(N * N, dtype=np.int32)                     # every ordered pair its own class
    m = make_model(orc, K, U, dtau, L, L)
    Z = 0.0
    acc = np.zeros((N * N, 4))
    per_config_gap = 0.0
    for bits in itertools.product((-1, 1), repeat=N * L):
        f = np.array(bits, dtype=np.int8).reshape(L, N)
        G0, ld0, s0 = orc.green_udv(m, f, 0, 0)
        G1, ld1, s1 = orc.green_udv(m, f, 1, 0)
        w = s0 * s1 * math.exp(ld0 + ld1)
        c = orc.correlations(np.stack([G0, G1]), cls, N * N)
        per_config_gap = max(per_config_gap, abs(c[1, 0] - 0.25 * (c[1, 2] + c[3, 2])))
        Z += w
        acc += w * c
    acc /= Z
    for x in range(N):
        for y in range(N):
            if x != y:
                assert acc[x * N + y, 0] == pytest.approx(0.25 * (acc[x * N + y, 2] + acc[y * N + x, 2]), abs=1e-12)
    assert per_config_gap > 1e-3


def test_translation_classes_partition_pairs():
    cls, n, r = W.translation_classes_square(4, 3)
    N = 12
    counts = np.bincount(cls, minlength=n)
    assert n == N and (counts == N).all() and r.shape == (N, 2)
    assert cls[0] == 0 and all(cls[i * N + i] == 0 for i in range(N))
    clsh, nh, _ = W.translation_classes_honeycomb(3, 2)
    assert nh == 24 and (np.bincount(clsh, minlength=nh) == 6).all()


def test_single_configuration_per_ordered_pair_equals_fock_trace(orc):
    """One field configuration, every ordered pair its own class, on a 3-site
    chain without reflection symmetry: the Wick values of orc_correlations on the
    configuration's G(0) equal Tr[O U_C] / Tr[U_C], U_C = U_L ... U_1 with
    U_tau = exp(-dtau H_T) exp(sum_s sum_i v^s_i,tau n_i,s) the configuration's
    Fock-space propagator (its G(0) = (1 + B(beta,0))^-1 is <c c+> of U_C).  Per
    configuration <S^+_x S^-_y> and <S^+_y S^-_x> differ, so this fixes the order
    of the two sites in each estimator, which the averages over all fields (real
    and symmetric) cannot."""
    from scipy.linalg import expm
    N, U, dtau, L = 3, 4.0, 0.2, 4
    K = W.chain_lattice(N, t=1.0, mu=0.2)
    K[0, 0] -= 0.4
    K[1, 2] = K[2, 1] = -0.7
    om = make_model(orc, K, U, dtau, L, 2)
    lam = math.acosh(math.exp(0.5 * dtau * U))
    F = Fock(N)
    ET = expm(-dtau * F.hopping(K))
    cls = np.arange(N * N, dtype=np.int32)
    for seed in (1, 2):
        f = np.where(np.random.default_rng(seed).random((L, N)) < 0.5, -1, 1).astype(np.int8)
        Uc = np.eye(F.dim)
        for t in range(L):
            V = sum(lam * f[t, i] * (F.n(0, i) - F.n(1, i)) for i in range(N))
            Uc = ET @ expm(V) @ Uc
        Z = np.trace(Uc)
        G = np.stack([orc.green_udv(om, f, s, 0)[0] for s in (0, 1)])
        got = orc.correlations(G, cls, N * N)
        cu = [F.c[F.mode(0, x)] for x in range(N)]
        cd = [F.c[F.mode(1, x)] for x in range(N)]
        for x in range(N):
            for y in range(N):
                szx, szy = 0.5 * (F.n(0, x) - F.n(1, x)), 0.5 * (F.n(0, y) - F.n(1, y))
                nx, ny = F.n(0, x) + F.n(1, x), F.n(0, y) + F.n(1, y)
                ops = (szx @ szy, nx @ ny, cu[x].T @ cd[x] @ cd[y].T @ cu[y], cu[x].T @ cu[y] + cd[x].T @ cd[y])
                want = [np.trace(O @ Uc) / Z for O in ops]
                assert np.abs(got[x * N + y] - want).max() < 1e-10, (seed, x, y, got[x * N + y], want)
        # the pin has power: per configuration the S^+ S^- estimator is not symmetric in x, y
        assert abs(got[0 * N + 2, 2] - got[2 * N + 0, 2]) > 1e-3
