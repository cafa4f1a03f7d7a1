"""The bin driver and the lattice analysis end to end on real Markov chains (CPU).

The measurement calls the bin driver makes (sweep, the energy window, equal-time
correlations per pair class) are served here by chains of the FP64 oracle,
which is test infrastructure: this checks the host pipeline -- bins over chains
and sweeps, sign reweighting, the delete-1 jackknife and the R -> K transform
with its background -- on Monte Carlo data, against exact diagonalisation of
the Trotterised density matrix of the 2 x 2 plaquette.  The reference S(k) is
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

    def measure_corr(self, classes, n_class):
        cls, nc = classes[0], int(n_class[0])
        out = np.stack([self.orc.correlations(np.stack([ch.green(0), ch.green(1)]), cls, nc) for ch in self.chains])
        sign = np.array([ch.fields()[2] for ch in self.chains], dtype=np.int32)
        return out, sign


def _ed_structure_factors(K, U, dtau, L, pos, k):
    """S^zz(k) and S^nn(k) (background subtracted) of the Trotterised density
    matrix, from the expectation of every site pair."""
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
    ph = np.exp(1j * (k @ pos.T))                                       # [n_k, N]: e^{i k R_x}
    S = lambda M: np.einsum("kx,xy,ky->k", ph.conj(), M, ph) / N       # (1/N) sum_xy e^{i k (R_y - R_x)} M_xy
    return S(Mzz), S(Mnn)


def test_bin_driver_structure_factors_match_exact_diagonalisation(orc):
    K = W.square_lattice(2, 2, t=1.0)
    U, dtau, L = 4.0, 0.125, 8
    m = W.ModelSpec(K, U=U, dtau=dtau, L=L, n_wrap=4)
    cls, ncls, r = W.translation_classes_square(2, 2)
    a1, a2 = np.array([1.0, 0.0]), np.array([0.0, 1.0])
    ens = OracleEnsemble(orc, m, n_chains=64, seed=91)
    res = Simulation(ens, n_bins=12, sweeps_per_bin=20, warmup=20, corr=([cls], [ncls]),
                     lattice=(a1, a2, 2 * a1, 2 * a2, 1, r)).run()
    k = res.mean["k"]
    pos = np.array([[x % 2, x // 2] for x in range(4)], dtype=float)
    zz_ed, nn_ed = _ed_structure_factors(K, U, dtau, L, pos, k)
    assert res.mean_sign == pytest.approx(1.0)
    F = Fock(4)
    rho = F.trotter_ising(K, U, dtau, L)
    kin_ed = np.trace(F.hopping(K) @ rho) / np.trace(rho)
    assert abs(res.mean["kin"] - kin_ed) < 5 * res.error["kin"]
    for name, ed in (("corr_zz_k", zz_ed), ("corr_nn_k", nn_ed)):
        mc, err = res.mean[name][:, 0, 0], res.error[name][:, 0, 0]
        assert np.abs(mc.imag).max() < 1e-12 and np.abs(ed.imag).max() < 1e-12
        z = np.abs(mc.real - ed.real) / (err.real + 1e-12)
        assert (z < 5.0).all(), (name, mc.real, err.real, ed.real)
    # the power of the check: S^zz at (pi, pi) is the largest and well resolved
    q = int(np.argmin(np.abs(k - np.pi).sum(axis=1)))
    assert res.mean["corr_zz_k"][q, 0, 0].real > 5 * res.error["corr_zz_k"][q, 0, 0].real
    assert zz_ed[q].real == max(zz_ed.real)
