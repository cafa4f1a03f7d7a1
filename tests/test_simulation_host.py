"""Bin bookkeeping of the Simulation driver, on a fake ensemble (no GPU)."""
import numpy as np
import pytest

from paper_1704_00131_gb300.simulation import Simulation


def _jack_mean(num, den, n_bins, f=lambda x: x):
    """Eq. jack_mean written out: the per-sweep sign-weighted sums num [sweeps, ...]
    and signs den [sweeps] grouped into n_bins consecutive bins, then the mean over
    i of f(sum_{b != i} num_b / sum_{b != i} den_b)."""
    nb = np.array_split(np.asarray(num, dtype=np.float64), n_bins)
    db = np.array_split(np.asarray(den, dtype=np.float64), n_bins)
    out = []
    for i in range(n_bins):
        N = sum(x.sum(axis=0) for b, x in enumerate(nb) if b != i)
        D = sum(x.sum() for b, x in enumerate(db) if b != i)
        out.append(f(N / D))
    return np.mean(out, axis=0)


class _Model:
    N = 4


class FakeEnsemble:
    """Deterministic stand-in with the measurement calls of dqmc.Ensemble."""

    def __init__(self, n_chains=3, L=4, seed=0, n_class=2):
        self.n_chains = n_chains
        self.n_class = n_class
        self.L = L
        self.seed = seed
        self.counter = 0                                # sweeps done: the random numbers follow from it
        self.fields = [np.ones((L, 4), dtype=np.int8) for _ in range(n_chains)]
        self.e = np.zeros((n_chains, 4))
        self.ss = np.zeros(n_chains)
        self.nm = np.zeros(n_chains, dtype=np.int64)
        self.log = []                                   # (sign, obs, corr) per sweep
        self.log_tau = []                               # time-displaced class sums per sweep

    def model_of(self, c):
        return _Model()

    def get_fields(self):
        return [f.copy() for f in self.fields], self.counter

    def set_fields(self, fields, counter):
        self.fields = [np.asarray(f, dtype=np.int8).copy() for f in fields]
        self.counter = counter

    def sweep(self, n, stats=False):
        for _ in range(n):
            rng = np.random.default_rng([self.seed, self.counter])
            self.counter += 1
            for f in self.fields:
                f[rng.integers(self.L), rng.integers(4)] *= -1
            sg = np.where(rng.random((self.n_chains, 2)) < 0.9, 1, -1).astype(np.int32)
            obs = rng.random((self.n_chains, self.L + 1, 2, 3))
            corr = rng.random((self.n_chains, self.n_class, 4))
            en = rng.random((self.n_chains, 4))
            s = np.prod(sg, axis=1)
            self.e += 2 * s[:, None] * en                   # two measurements per sweep
            self.ss += 2 * s
            self.nm += 2
            self.log.append((s.astype(float), obs, corr, en))
            self.cur = (sg, obs, corr)

    def measure(self):
        return self.e.copy(), self.ss.copy(), self.nm.copy()

    def measure_tau(self, n_tau, phases):
        sg, obs, _ = self.cur
        return obs, sg, np.zeros(2)

    def measure_tau_corr(self, n_tau, classes, n_class):
        sg, obs, corr = self.cur
        rng = np.random.default_rng([self.seed, self.counter, 7])
        out = rng.random((self.n_chains, n_tau + 1, self.n_class, 3))
        self.log_tau.append(out)
        return out, np.prod(sg, axis=1).astype(np.int32)

    def measure_corr(self, classes, n_class):
        sg, _, corr = self.cur
        return corr, np.prod(sg, axis=1).astype(np.int32)


def test_bins_pool_chains_and_reweight_by_sign():
    ens = FakeEnsemble()
    sim = Simulation(ens, n_bins=4, sweeps_per_bin=5, warmup=2, tau=(4, None), corr=([None], [2]))
    res = sim.run()
    log = ens.log[2:]                                   # after the warm-up
    s = np.array([x[0] for x in log])                   # [sweeps, chains]
    corr = np.array([x[2] for x in log])                # [sweeps, chains, class, 4]
    en = np.array([x[3] for x in log])
    ss = s.sum(axis=1)                                  # sign summed over chains, per sweep
    want_zz = _jack_mean((s[:, :, None] * corr[:, :, :, 0]).sum(axis=1), ss, 4)
    assert res.mean["corr_zz"] == pytest.approx(want_zz, rel=1e-12)
    # a bin's reweighted ratio sits close to the pooled one (the estimate differs by the jackknife's O(1/N_bin))
    assert res.mean["corr_zz"] == pytest.approx((s[:, :, None] * corr[:, :, :, 0]).sum(axis=(0, 1)) / s.sum(), rel=0.05)
    want_kin = _jack_mean((s * en[:, :, 0]).sum(axis=1), ss, 4)
    assert res.mean["kin"] == pytest.approx(want_kin, rel=1e-12)
    obs = np.array([x[1] for x in log])                 # [sweeps, chains, tau, fl, 3]
    m = obs[..., 0, 2] - obs[..., 1, 2]
    szz = (m * m[..., :1] + obs[..., 0, 1] + obs[..., 1, 1]) / 4.0
    want_szz = _jack_mean((s[:, :, None] * szz).sum(axis=1), ss, 4)
    assert res.mean["szz_tau"] == pytest.approx(want_szz, rel=1e-12)
    gl = obs[..., 0].sum(axis=3) / (2 * 4)
    assert res.mean["gloc_tau"] == pytest.approx(_jack_mean((s[:, :, None] * gl).sum(axis=1), ss, 4), rel=1e-12)
    assert all(np.all(np.asarray(res.error[k]) > 0) for k in res.mean)
    assert res.mean_sign == pytest.approx(s.mean(), rel=1e-12)
    assert res.n_bins == 4 and res.sweeps_per_bin == 5


def test_bad_parameters():
    with pytest.raises(ValueError):
        Simulation(FakeEnsemble(), n_bins=1, sweeps_per_bin=1)
    with pytest.raises(ValueError):
        Simulation(FakeEnsemble(), n_bins=2, sweeps_per_bin=0)


def test_checkpoint_resume_equals_uninterrupted_run(tmp_path):
    kw = dict(n_bins=5, sweeps_per_bin=3, warmup=2, tau=(4, None), corr=([None], [2]))
    full = Simulation(FakeEnsemble(seed=7), **kw).run()
    path = str(tmp_path / "run.npz")
    part = Simulation(FakeEnsemble(seed=7), **kw).run(checkpoint=path, max_seconds=0.0)
    assert not part.complete and part.mean == {}         # stopped after the first bin
    ens = FakeEnsemble(seed=7)
    resumed = Simulation(ens, **kw).run(checkpoint=path)
    assert resumed.complete and ens.counter == 2 + 5 * 3
    assert resumed.mean_sign == full.mean_sign
    for k in full.mean:
        if k in ("kin", "pot", "part", "ener"):
            # differences of running sums that restart from zero on the fresh ensemble: equal to rounding
            assert resumed.mean[k] == pytest.approx(full.mean[k], rel=1e-12), k
            assert resumed.error[k] == pytest.approx(full.error[k], rel=1e-12), k
        else:
            assert np.array_equal(resumed.mean[k], full.mean[k]) and np.array_equal(resumed.error[k], full.error[k]), k
    # a finished checkpoint resumes to the same result without sweeping
    ens2 = FakeEnsemble(seed=7)
    again = Simulation(ens2, **kw).run(checkpoint=path)
    assert ens2.counter == 2 + 5 * 3 and np.array_equal(again.mean["corr_zz"], full.mean["corr_zz"])
    f_end, _ = ens.get_fields()
    assert all(np.array_equal(a, b) for a, b in zip(ens2.get_fields()[0], f_end))


def test_checkpoint_of_another_run_is_rejected(tmp_path):
    path = str(tmp_path / "run.npz")
    Simulation(FakeEnsemble(), n_bins=3, sweeps_per_bin=2).run(checkpoint=path)
    with pytest.raises(ValueError):
        Simulation(FakeEnsemble(), n_bins=4, sweeps_per_bin=2).run(checkpoint=path)
    with pytest.raises(ValueError):
        Simulation(FakeEnsemble(n_chains=2), n_bins=3, sweeps_per_bin=2).run(checkpoint=path)


def test_lattice_resolved_structure_factors():
    """With a lattice the bin driver turns the per-class correlation bins into
    S_ab(k): the sign-reweighted pooled class sums through analysis.structure_factor,
    the density's background from the local sum_s <c+ c> at d = 0."""
    from paper_1704_00131_gb300 import analysis as A
    from paper_1704_00131_gb300 import workloads as W
    L1, L2 = 2, 2
    cls, ncls, r = W.translation_classes_honeycomb(L1, L2)
    a1, a2 = np.array([1.0, 0.0]), np.array([0.5, np.sqrt(3.0) / 2.0])
    ens = FakeEnsemble(n_class=ncls)
    sim = Simulation(ens, n_bins=4, sweeps_per_bin=3, corr=([cls], [ncls]), lattice=(a1, a2, L1 * a1, L2 * a2, 2, r))
    res = sim.run()
    s = np.array([x[0] for x in ens.log])                   # [sweeps, chains]
    corr = np.array([x[2] for x in ens.log])                # [sweeps, chains, class, 4]
    k = A.momenta(a1, a2, L1 * a1, L2 * a2)
    assert np.abs(res.mean["k"] - k).max() == 0.0
    num = (s[:, :, None, None] * corr).sum(axis=1)
    want_nn = _jack_mean(num, s.sum(axis=1), 4, lambda p: A.structure_factor(
        p[:, 1], r, a1, a2, k, L1 * L2, 2, O_mean=p[[0, 3], 3] / (L1 * L2)))
    want_zz = _jack_mean(num, s.sum(axis=1), 4, lambda p: A.structure_factor(p[:, 0], r, a1, a2, k, L1 * L2, 2))
    assert np.abs(res.mean["corr_nn_k"] - want_nn).max() < 1e-12
    assert np.abs(res.mean["corr_zz_k"] - want_zz).max() < 1e-12
    assert res.error["corr_nn_k"].shape == want_nn.shape and np.all(res.error["corr_nn_k"].real > 0)
    with pytest.raises(ValueError):
        Simulation(ens, n_bins=4, sweeps_per_bin=3, lattice=(a1, a2, L1 * a1, L2 * a2, 2, r))


def test_time_displaced_structure_factors():
    """tau_corr with a lattice: S_ab(k, tau) of the three time-displaced
    correlations from the pooled class sums; the density's background from
    sum_s G(0,0)_xx = 2 - <n_x> at tau = 0."""
    from paper_1704_00131_gb300 import analysis as A
    from paper_1704_00131_gb300 import workloads as W
    L1, L2, n_tau = 2, 2, 3
    cls, ncls, r = W.translation_classes_honeycomb(L1, L2)
    a1, a2 = np.array([1.0, 0.0]), np.array([0.5, np.sqrt(3.0) / 2.0])
    ens = FakeEnsemble(n_class=ncls)
    sim = Simulation(ens, n_bins=3, sweeps_per_bin=2, energy=False, tau_corr=(n_tau, [cls], [ncls]),
                     lattice=(a1, a2, L1 * a1, L2 * a2, 2, r), n_cov=True)
    res = sim.run()
    s = np.array([x[0] for x in ens.log])                   # [sweeps, chains]
    o = np.array(ens.log_tau)                               # [sweeps, chains, tau, class, 3]
    k = A.momenta(a1, a2, L1 * a1, L2 * a2)
    num = (s[:, :, None, None, None] * o).sum(axis=1)
    want_nn = _jack_mean(num, s.sum(axis=1), 3, lambda p: A.structure_factor(
        p[..., 2], r, a1, a2, k, L1 * L2, 2, O_mean=2.0 - p[0, [0, 3], 0] / (L1 * L2)))
    want_gf = _jack_mean(num, s.sum(axis=1), 3, lambda p: A.structure_factor(p[..., 0], r, a1, a2, k, L1 * L2, 2))
    assert res.mean["nn_tau_k"].shape == (n_tau + 1, L1 * L2, 2, 2)
    assert np.abs(res.mean["nn_tau_k"] - want_nn).max() < 1e-12
    assert np.abs(res.mean["gf_tau_k"] - want_gf).max() < 1e-12
    assert "szz_tau_k" in res.error and res.mean_sign != 0.0
    c = res.cov["nn_tau_k"]
    assert c.shape == (n_tau + 1, n_tau + 1, L1 * L2, 2, 2)
    assert np.abs(np.einsum("ttkab->tkab", c) - res.error["nn_tau_k"].real ** 2).max() < 1e-12


def test_skip_and_rebin_bins():
    """n_skip drops the first bins and n_rebin merges consecutive ones before the
    jackknife: 6 bins of 2 sweeps with n_skip = 2, n_rebin = 2 analyse as 2 bins of
    4 sweeps starting at the fifth sweep."""
    ens = FakeEnsemble()
    res = Simulation(ens, n_bins=6, sweeps_per_bin=2, corr=([None], [2]), n_skip=2, n_rebin=2, energy=False).run()
    log = ens.log[4:]
    s = np.array([x[0] for x in log])
    corr = np.array([x[2] for x in log])
    want = _jack_mean((s[:, :, None] * corr[:, :, :, 1]).sum(axis=1), s.sum(axis=1), 2)
    assert res.mean["corr_nn"] == pytest.approx(want, rel=1e-12)
    with pytest.raises(ValueError):
        Simulation(ens, n_bins=4, sweeps_per_bin=2, n_skip=1, n_rebin=2)
