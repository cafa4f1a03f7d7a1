"""The GPU's time-displaced and equal-time measurements, sampled by the GPU's own
Markov chains, against exact diagonalisation of the Trotterised 2x2 Hubbard
plaquette (Fock-space traces with the operators inserted between Trotter
factors).  64 independent chains; the error of each average is the spread of
the per-chain means, and every quantity must agree within 4 sigma (about 70
comparisons: a 3-sigma bar would trip by chance in one run of six).  Seeds
are fixed and the kernels deterministic, so the outcome is reproducible.
"""
import numpy as np
import pytest

from paper_1704_00131_gb300 import analysis as A
from paper_1704_00131_gb300 import workloads as W

from .fock_ed import Fock, equal_time_correlations, tau_observables

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00131_gb300 import build_ext, dqmc
    build_ext.build()
    return dqmc


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_measurements_match_exact_diagonalisation(dq, precision):
    K = W.square_lattice(2, 2, t=1.0)
    U, dtau, L = 4.0, 0.125, 8
    m = W.ModelSpec(K, U=U, dtau=dtau, L=L, n_wrap=4)
    ph = W.sublattice_signs_square(2, 2)
    cls, ncls, _ = W.translation_classes_square(2, 2)
    F = Fock(4)
    gl_ed, szz_ed = tau_observables(F, K, U, dtau, L, ph)
    corr_ed = equal_time_correlations(F, K, U, dtau, L, cls, ncls)

    n_chains, n_sweeps = 64, 120
    ens = dq.Ensemble([m], [0] * n_chains, precision=precision, seed=77)
    ens.sweep(20, stats=False)
    s_sum = np.zeros(n_chains)
    gl_sum = np.zeros((n_chains, L + 1))
    szz_sum = np.zeros((n_chains, L + 1))
    corr_sum = np.zeros((n_chains, ncls, 4))
    for _ in range(n_sweeps):
        ens.sweep(1, stats=False)
        obs, sg, _ = ens.measure_tau(L, [ph])
        w = np.prod(sg, axis=1).astype(float)                    # configuration sign
        corr, sgc = ens.measure_corr([cls], [ncls])
        assert np.array_equal(sgc, w.astype(np.int32))
        s_sum += w
        gl_sum += w[:, None] * (obs[:, :, 0, 0] + obs[:, :, 1, 0])
        szz_sum += w[:, None] * dq.szz_tau(obs)
        corr_sum += w[:, None, None] * corr
    ens.close()

    def check(per_chain_os, ref, what):
        # per-chain means of O s and s as jackknife bins
        mean, err = A.jackknife(per_chain_os / n_sweeps, s_sum / n_sweeps)
        z = np.abs(mean - ref) / (err + 1e-12)
        assert (z < 4.0).all(), (what, mean, err, ref)

    check(gl_sum, gl_ed, "local G(tau)")
    check(szz_sum, szz_ed, "staggered S^z S^z(tau)")
    check(corr_sum.reshape(n_chains, -1), corr_ed.ravel(), "equal-time correlations")
    # the equal-time slice of the displaced measurement and the correlation
    # function measure the same staggered S^z S^z
    stag = np.array([ph[0] * ph[j] for j in range(4)])
    assert np.allclose(szz_sum[:, 0], (corr_sum[:, :, 0] * stag[None, :]).sum(axis=1), atol=1e-6)


def test_simulation_driver_matches_exact_diagonalisation(dq):
    """The bin driver over the same calls: energy (measurement window), local
    G(tau) and the equal-time correlations, jackknife over 8 bins (whose error
    bars are themselves uncertain by about a quarter), within 5 sigma."""
    from paper_1704_00131_gb300.simulation import Simulation
    K = W.square_lattice(2, 2, t=1.0)
    U, dtau, L = 4.0, 0.125, 8
    m = W.ModelSpec(K, U=U, dtau=dtau, L=L, n_wrap=4)
    cls, ncls, _ = W.translation_classes_square(2, 2)
    F = Fock(4)
    gl_ed, _ = tau_observables(F, K, U, dtau, L, np.ones(4))
    corr_ed = equal_time_correlations(F, K, U, dtau, L, cls, ncls)
    rho = F.trotter_ising(K, U, dtau, L)
    kin_ed = np.trace(F.hopping(K) @ rho) / np.trace(rho)
    ens = dq.Ensemble([m], [0] * 32, precision="fp64", seed=404, measure=True, meas_first=0, meas_last=L)
    res = Simulation(ens, n_bins=8, sweeps_per_bin=15, warmup=20, tau=(L, None), corr=([cls], [ncls])).run()
    ens.close()
    assert res.mean_sign == pytest.approx(1.0)
    # per-chain averages: kin per measurement, gloc per site and flavor (8 = 2 x 4)
    assert abs(res.mean["kin"] - kin_ed) < 5 * res.error["kin"] + 1e-12
    assert (np.abs(res.mean["gloc_tau"] * 8 - gl_ed) < 5 * res.error["gloc_tau"] * 8 + 1e-12).all()
    assert (np.abs(res.mean["corr_zz"] - corr_ed[:, 0]) < 5 * res.error["corr_zz"] + 1e-12).all()
