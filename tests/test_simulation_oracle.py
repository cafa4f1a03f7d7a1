"""The bin driver and the lattice analysis end to end on real Markov chains (CPU).

The measurement calls the bin driver makes (sweep, the energy window, equal-time
correlations per pair class) are served here by chains of the FP64 oracle,
which is test infrastructure: this checks the host pipeline -- bins over chains
and sweeps, sign reweighting, the delete-1 jackknife and the R -> K transform
with its background -- on Monte Carlo data, against exact diagonalisation of
the Trotterised density matrix of the 2 x 2 plaquette and of a 2 x 1 honeycomb
(two orbitals per cell, 2 x 2 matrices S_ab(k)).  The reference S(k) is
the plain definition (1/N) sum_xy e^{i k (R_y - R_x)} (<O_x O_y> - <O_x><O_y>)
over all site pairs, not the per-class path the driver takes.
"""
import numpy as np
import pytest

from paper_1704_00131_gb300 import workloads as W
from paper_1704_00131_gb300.simulation import Simulation

from .fock_ed import Fock


class OracleEnsemble:
    """The calls of dqmc.Ensemble that Simulation makes, on oracle chains."""

    def __init__(self, orc, m: W.ModelSpec, n_chains: int, seed: int):
        self.orc = orc
        self.m = m
        om = orc.Model(m.hopping, m.vertex_site, m.vertex_sign, m.U, m.dtau, m.L, m.n_wrap, m.field_type)
        self.om = om
        self.chains = [orc.Chain(om, None, seed=seed, chain=c, measure=True) for c in range(n_chains)]
        self.n_chains = n_chains

    def model_of(self, c):
        return self.m

    def sweep(self, n, stats=False):
        for ch in self.chains:
            ch.sweep(n)

    def measure(self):
        r = [ch.measure() for ch in self.chains]
        return (np.array([x[0] for x in r]), np.array([x[1] for x in r]), np.array([x[2] for x in r]))

    def measure_tau_corr(self, n_tau, classes, n_class):
        cls, nc = classes[0], int(n_class[0])
        out = np.stack([self.orc.tau_correlations(self.om, ch.fields()[0], n_tau, cls, nc) for ch in self.chains])
        sign = np.array([ch.fields()[2] for ch in self.chains], dtype=np.int32)
        return out, sign

    def measure_corr(self, classes, n_class):
        cls, nc = classes[0], int(n_class[0])
        out = np.stack([self.orc.correlations(np.stack([ch.green(0), ch.green(1)]), cls, nc) for ch in self.chains])
        sign = np.array([ch.fields()[2] for ch in self.chains], dtype=np.int32)
        return out, sign


def _ed_structure_factors(K, U, dtau, L, cell_pos, n_orb, k):
    """S^zz_ab(k) and S^nn_ab(k) (background subtracted) of the Trotterised density
    matrix, from the expectation of every site pair: site x = n_orb cell + orbital,
    S_ab(k) = (1/N_cell) sum_ij e^{i k (R_j - R_i)} (<O_ia O_jb> - <O_ia><O_jb>)."""
    N = K.shape[0]
    F = Fock(N)
    rho = F.trotter_ising(K, U, dtau, L)
    Z = np.trace(rho)
    sz = [0.5 * (F.n(0, x) - F.n(1, x)) for x in range(N)]
    nn = [F.n(0, x) + F.n(1, x) for x in range(N)]
    ev = lambda O: np.trace(O @ rho) / Z
    Mzz = np.array([[ev(sz[x] @ sz[y]) for y in range(N)] for x in range(N)])
    n1 = np.array([ev(nn[x]) for x in range(N)])
    Mnn = np.array([[ev(nn[x] @ nn[y]) for y in range(N)] for x in range(N)]) - np.outer(n1, n1)
    n_cells = N // n_orb
    ph = np.exp(1j * (k @ cell_pos.T))                                  # [n_k, N_cell]: e^{i k R_i}

    def S(M):
        Mc = M.reshape(n_cells, n_orb, n_cells, n_orb)                  # [i, a, j, b]
        return np.einsum("ki,iajb,kj->kab", ph.conj(), Mc, ph) / n_cells

    return S(Mzz), S(Mnn)


A1, A2SQ, A2H = np.array([1.0, 0.0]), np.array([0.0, 1.0]), np.array([0.5, np.sqrt(3.0) / 2.0])
CASES = {
    # name: (hopping, classes, unit vectors, periodicity in cells, orbitals)
    "square2x2": (lambda: W.square_lattice(2, 2, t=1.0), lambda: W.translation_classes_square(2, 2), A2SQ, (2, 2), 1),
    "honeycomb2x1": (lambda: W.honeycomb_lattice(2, 1, t=1.0), lambda: W.translation_classes_honeycomb(2, 1), A2H,
                     (2, 1), 2),
}


@pytest.mark.parametrize("case", list(CASES))
def test_bin_driver_structure_factors_match_exact_diagonalisation(orc, case):
    hop, classes, a2, (l1, l2), n_orb = CASES[case]
    K = hop()
    U, dtau, L = 4.0, 0.125, 8
    m = W.ModelSpec(K, U=U, dtau=dtau, L=L, n_wrap=4)
    cls, ncls, r = classes()
    ens = OracleEnsemble(orc, m, n_chains=64, seed=91)
    res = Simulation(ens, n_bins=12, sweeps_per_bin=20, warmup=20, corr=([cls], [ncls]),
                     lattice=(A1, a2, l1 * A1, l2 * a2, n_orb, r)).run()
    k = res.mean["k"]
    n_cells = l1 * l2
    cell_pos = np.array([(c % l1) * A1 + (c // l1) * a2 for c in range(n_cells)])
    zz_ed, nn_ed = _ed_structure_factors(K, U, dtau, L, cell_pos, n_orb, k)
    assert res.mean_sign == pytest.approx(1.0)
    F = Fock(K.shape[0])
    rho = F.trotter_ising(K, U, dtau, L)
    kin_ed = np.trace(F.hopping(K) @ rho) / np.trace(rho)
    assert abs(res.mean["kin"] - kin_ed) < 5 * res.error["kin"]
    for name, ed in (("corr_zz_k", zz_ed), ("corr_nn_k", nn_ed)):
        mc, err = res.mean[name], res.error[name]
        for part, e in ((np.real, err.real), (np.imag, err.imag)):
            z = np.abs(part(mc) - part(ed)) / (e + 1e-12)
            assert (z < 5.0).all(), (name, mc, err, ed)
    # the power of the check: the largest S^zz component is resolved
    q, a, b = np.unravel_index(np.argmax(zz_ed.real), zz_ed.shape)
    assert res.mean["corr_zz_k"][q, a, b].real > 5 * res.error["corr_zz_k"][q, a, b].real


def test_bin_driver_time_displaced_structure_factors_match_exact_diagonalisation(orc):
    """tau_corr: S^zz(k, tau) and the background-subtracted S^nn(k, tau) of the 2 x 2
    plaquette for every tau against <A(tau) B(0)> = Tr[T^(L-tau) A T^tau B] / Tr[T^L]
    of every site pair, T the Trotter factor of one slice."""
    from scipy.linalg import expm
    K = W.square_lattice(2, 2, t=1.0)
    U, dtau, L = 4.0, 0.125, 8
    m = W.ModelSpec(K, U=U, dtau=dtau, L=L, n_wrap=4)
    cls, ncls, r = W.translation_classes_square(2, 2)
    ens = OracleEnsemble(orc, m, n_chains=64, seed=92)
    res = Simulation(ens, n_bins=12, sweeps_per_bin=20, warmup=20, tau_corr=(L, [cls], [ncls]), energy=False,
                     lattice=(A1, A2SQ, 2 * A1, 2 * A2SQ, 1, r), n_cov=True).run()
    k = res.mean["k"]
    N = 4
    F = Fock(N)
    T = expm(-dtau * F.hopping(K)) @ expm(-dtau * F.hubbard_ph(U))
    Z = np.trace(np.linalg.matrix_power(T, L))
    sz = [0.5 * (F.n(0, x) - F.n(1, x)) for x in range(N)]
    nn = [F.n(0, x) + F.n(1, x) for x in range(N)]
    n1 = np.array([np.trace(np.linalg.matrix_power(T, L) @ nn[x]) / Z for x in range(N)])
    pos = np.array([[x % 2, x // 2] for x in range(N)], dtype=float)
    ph = np.exp(1j * (k @ pos.T))
    for tau in range(L + 1):
        Aa, Bb = np.linalg.matrix_power(T, L - tau), np.linalg.matrix_power(T, tau)
        Mzz = np.array([[np.trace(Aa @ sz[x] @ Bb @ sz[y]) / Z for y in range(N)] for x in range(N)])
        Mnn = np.array([[np.trace(Aa @ nn[x] @ Bb @ nn[y]) / Z for y in range(N)] for x in range(N)]) - np.outer(n1, n1)
        for name, M in (("szz_tau_k", Mzz), ("nn_tau_k", Mnn)):
            ed = np.einsum("kx,xy,ky->k", ph.conj(), M, ph) / N
            mc, err = res.mean[name][tau, :, 0, 0], res.error[name][tau, :, 0, 0]
            z = np.abs(mc.real - ed.real) / (err.real + 1e-12)
            assert (z < 5.0).all(), (name, tau, mc.real, err.real, ed.real)
    # neighbouring imaginary times are correlated: positive covariance between tau and tau + 1
    c = res.cov["szz_tau_k"][:, :, 3, 0, 0]
    assert c[4, 5] > 0 and np.allclose(np.diag(c), res.error["szz_tau_k"][:, 3, 0, 0].real ** 2)
