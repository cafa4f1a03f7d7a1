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
