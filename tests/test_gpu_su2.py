"""The SU(2) charge decoupling on the GPU (dqmc_su2_*: complex FP64, one CTA per
chain) against the oracle (Sec. 6.1 model; Sec. 2.1 transform with imaginary
coupling; Sec. 2.2 phase; Sec. 2.3 stabilisation).

* Fields drawn by the library equal the oracle's Philox draws bit for bit.
* Fixed fields: G(0), log|det(1 + B)| and arg det(1 + B) of the complex UDV
  chain against orc_su2_green_udv (FP64: 1e-10) at beta = 2 and at the paper's
  example beta = 10 (4 x 4, U = 4, n_wrap = 10), at and away from half filling;
  the phase P = exp(i (-g sum eta + 2 arg det)).
* Markov chain: the field trajectory, acceptance count and phase after each
  sweep equal orc_su2_sweep (plain recompute of G~ for every proposal) on the
  same Philox streams, and the reweighted energy at tau = 0 agrees.
* Precision Green / Precision Phase at beta = 10 stay at the level of the
  paper's example; at half filling every weight is positive (sign 1, P = 1).
* Hubbard-Ising bond model (Sec. 6): Ising spins on bonds entering the
  propagator as two-site factors; G(0), log|det| and arg det against the
  oracle's bond-model UDV chain, and the joint trajectory of HS fields and bond
  spins (rank-2 updates, the spins' own weight) against its Markov chain.
"""
import numpy as np
import pytest

from paper_1704_00131_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00131_gb300 import build_ext, dqmc
    build_ext.build()
    return dqmc


def _wrap(a):
    return (a + np.pi) % (2 * np.pi) - np.pi


def _phase(orc, f, dtau, U, ar):
    g = np.sqrt(0.5 * dtau * U)
    ph = -g * sum(orc.field_coupling(2, 1.0, 2.0, int(l)) for l in np.asarray(f).ravel())
    return np.exp(1j * (ph + 2.0 * ar))


def test_su2_fields_drawn_like_the_oracle(dq, orc):
    m = dq.Su2Model(W.square_lattice(4, 4), U=4.0, dtau=0.1, L=20, n_wrap=5)
    ens = dq.Su2Ensemble([m], [0, 0, 0], seed=777)
    fields, ctr = ens.get_fields()
    assert ctr == 0
    for c in range(3):
        ref = np.asarray(orc.init_fields(2, m.L, m.N, 777, c)).reshape(m.L, m.N)
        assert np.array_equal(fields[c], ref), c
    ens.close()


@pytest.mark.parametrize("mu,L,nw", [(0.0, 20, 5), (0.3, 20, 5), (0.0, 100, 10), (-0.5, 100, 10)])
def test_su2_fresh_green_matches_oracle(dq, orc, mu, L, nw):
    K = W.square_lattice(4, 4, t=1.0, mu=mu)
    dtau, U = 0.1, 4.0
    rng = np.random.default_rng(int(L + 100 * mu))
    fields = [rng.choice([-2, -1, 1, 2], size=(L, 16)).astype(np.int8) for _ in range(3)]
    m = dq.Su2Model(K, U=U, dtau=dtau, L=L, n_wrap=nw)
    ens = dq.Su2Ensemble([m], [0, 0, 0], fields=fields, seed=5)
    for c in range(3):
        Go, lo, ao = orc.su2_green_udv(K, dtau, U, nw, fields[c], 0)
        for fresh in (False, True):
            G, la, ar, P = ens.greens(c, fresh=fresh)
            assert np.abs(G - Go).max() < 1e-10, (c, fresh)
            assert la == pytest.approx(lo, rel=1e-10, abs=1e-10)
            assert abs(_wrap(ar - ao)) < 1e-10
            assert abs(P - _phase(orc, fields[c], dtau, U, ao)) < 1e-9
        if L == 20:   # small beta: also the plain product
            Gp, lp, ap, _, _, _ = orc.su2_plain(K, dtau, U, fields[c])
            assert np.abs(G - Gp).max() < 1e-10 and abs(_wrap(ar - ap)) < 1e-10
    ens.close()


@pytest.mark.parametrize("lattice,mu", [("plaquette", 0.0), ("plaquette", 0.4), ("square4", 0.0), ("square4", -0.3)])
def test_su2_trajectory_matches_oracle(dq, orc, lattice, mu):
    """Three sweeps of four chains: fields, acceptances, phase and the reweighted
    energy at tau = 0 against the oracle's chain (plain recompute per proposal)."""
    if lattice == "plaquette":
        K, dtau, U, L, nw, n_sweeps = W.square_lattice(2, 2, t=1.0, mu=mu), 0.125, 4.0, 8, 4, 3
    else:
        K, dtau, U, L, nw, n_sweeps = W.square_lattice(4, 4, t=1.0, mu=mu), 0.1, 4.0, 20, 5, 2
    N, seed, n_ch = K.shape[0], 2024, 4
    f0 = [np.asarray(orc.init_fields(2, L, N, 99, c), dtype=np.int8).reshape(L, N) for c in range(n_ch)]
    m = dq.Su2Model(K, U=U, dtau=dtau, L=L, n_wrap=nw)
    ens = dq.Su2Ensemble([m], [0] * n_ch, fields=f0, seed=seed, measure=True, meas_first=0, meas_last=0)
    chains = [orc.Su2Chain(K, dtau, U, f0[c], seed=seed, chain=c) for c in range(n_ch)]
    for sweep in range(n_sweeps):
        st = ens.sweep(1)
        obs, sg, nm = ens.measure(reset=True)
        fields, _ = ens.get_fields()
        acc = 0
        for c in range(n_ch):
            o, s_o, a = chains[c].sweep()
            acc += a
            assert np.array_equal(fields[c], chains[c].fields.reshape(L, N)), (sweep, c)
            _, _, _, P = ens.greens(c)
            Po = complex(chains[c].phase[0], chains[c].phase[1])
            assert abs(P - Po) < 1e-9, (sweep, c)
            assert nm[c] == 1 and sg[c] == s_o
            assert abs(obs[c, 3] - o) < 1e-8 * max(1.0, abs(o)), (sweep, c)
        assert st["accepted"] == acc and st["proposals"] == n_ch * 2 * L * N
        assert 0 < acc < st["proposals"]
    ens.close()


def test_su2_paper_example_precision(dq):
    """4 x 4, U = 4, beta = 10 (the paper's SU(2) example), n_wrap = 10, half
    filling: Precision Green / Phase at the level the paper reports for its
    example, sign 1 and a real phase throughout."""
    m = dq.Su2Model(W.square_lattice(4, 4), U=4.0, dtau=0.1, L=100, n_wrap=10)
    ens = dq.Su2Ensemble([m], [0] * 8, seed=11)
    ens.sweep(2)
    st = ens.sweep(3)
    assert st["prec_green_max"] < 1e-8 and st["prec_green_mean"] < 1e-10
    assert st["prec_phase_max"] < 1e-8
    assert st["mean_sign"] == 1.0
    assert 0.1 < st["accepted"] / st["proposals"] < 0.9
    for c in range(8):
        _, _, _, P = ens.greens(c)
        assert abs(P.imag) < 1e-8 and P.real > 0
    ens.close()


def test_su2_rejects_bad_input(dq):
    m = dq.Su2Model(W.square_lattice(2, 2), U=4.0, dtau=0.1, L=10, n_wrap=3)
    with pytest.raises(dq.DqmcError) as e:
        dq.Su2Ensemble([m], [0])
    assert e.value.status == dq.DQMC_EINVAL
    m = dq.Su2Model(W.square_lattice(2, 2), U=4.0, dtau=0.1, L=10, n_wrap=5)
    bad = np.ones((10, 4), dtype=np.int8)
    bad[3, 2] = 0
    with pytest.raises(dq.DqmcError) as e:
        dq.Su2Ensemble([m], [0], fields=[bad])
    assert e.value.status == dq.DQMC_EINVAL


# ------------------------------------------------ Hubbard-Ising bond model
def _square_bonds(Lx, Ly):
    idx = lambda x, y: (x % Lx) + Lx * (y % Ly)
    return [(idx(x, y), idx(x + 1, y)) for y in range(Ly) for x in range(Lx)] + \
           [(idx(x, y), idx(x, y + 1)) for y in range(Ly) for x in range(Lx)]


def _bond_config(rng, L, N, nb):
    hs = rng.choice(np.array([-2, -1, 1, 2], dtype=np.int8), size=(L, N))
    z = rng.choice(np.array([-1, 1], dtype=np.int8), size=(L, nb))
    return hs, z


@pytest.mark.parametrize("L,nw,mu", [(15, 5, 0.2), (100, 10, 0.3)])
def test_bond_model_fresh_green_matches_oracle(dq, orc, L, nw, mu):
    """3 x 3 square with an Ising spin on every bond: G(0), log|det| and arg det of
    the complex UDV chain with the bond factors against the oracle's chain."""
    K = W.square_lattice(3, 3, t=1.0, mu=mu)
    bonds = _square_bonds(3, 3)
    xi, h, J, dtau, U = 0.4, 0.6, 0.3, 0.1, 4.0
    pairs = [(b, (b + 1) % len(bonds)) for b in range(len(bonds))]
    rng = np.random.default_rng(L)
    cfg = [_bond_config(rng, L, 9, len(bonds)) for _ in range(2)]
    m = dq.Su2Model(K, U=U, dtau=dtau, L=L, n_wrap=nw, bonds=bonds, xi=xi, h=h, J=J, pairs=pairs)
    ens = dq.Su2Ensemble([m], [0, 0], fields=[np.concatenate([hs, z], axis=1) for hs, z in cfg], seed=1)
    for c, (hs, z) in enumerate(cfg):
        Go, lo, ao = orc.hubbard_ising_green_udv(K, bonds, xi, dtau, U, nw, hs, z, 0)
        for fresh in (False, True):
            G, la, ar, _ = ens.greens(c, fresh=fresh)
            assert np.abs(G - Go).max() < 1e-10, (c, fresh)
            assert la == pytest.approx(lo, rel=1e-10, abs=1e-10) and abs(_wrap(ar - ao)) < 1e-10
    f, _ = ens.get_fields()
    assert all(np.array_equal(f[c], np.concatenate(cfg[c], axis=1)) for c in range(2))
    ens.close()


@pytest.mark.parametrize("case", ["chain3_half", "chain3_mu", "square3x3"])
def test_bond_model_trajectory_matches_oracle(dq, orc, case):
    """HS fields and bond spins sampled together: after every sweep the fields,
    the spins, the acceptance count, the phase and the reweighted Kin and
    (sum_b s_b)^2 / n_bonds at tau = 0 equal the oracle's chain (plain recompute
    of the Green function at every vertex)."""
    if case.startswith("chain3"):
        K = W.chain_lattice(3, t=1.0, mu=0.0 if case == "chain3_half" else 0.4)
        bonds, pairs, L, nw, dtau, n_sweeps = [(0, 1), (1, 2)], [(0, 1)], 4, 2, 0.25, 3
        xi, h, J, U = 0.7, 0.8, 0.4, 2.0
    else:
        K = W.square_lattice(3, 3, t=1.0, mu=0.2)
        bonds = _square_bonds(3, 3)
        pairs = [(b, (b + 9) % 18) for b in range(9)]
        L, nw, dtau, n_sweeps = 8, 4, 0.125, 2
        xi, h, J, U = 0.4, 0.6, 0.3, 4.0
    N, nb, n_ch, seed = K.shape[0], len(bonds), 3, 4321
    rng = np.random.default_rng(7)
    cfg = [_bond_config(rng, L, N, nb) for _ in range(n_ch)]
    m = dq.Su2Model(K, U=U, dtau=dtau, L=L, n_wrap=nw, bonds=bonds, xi=xi, h=h, J=J, pairs=pairs)
    ens = dq.Su2Ensemble([m], [0] * n_ch, fields=[np.concatenate([hs, z], axis=1) for hs, z in cfg], seed=seed,
                         measure=True, meas_first=0, meas_last=0)
    chains = [orc.HubbardIsingChain(K, bonds, xi, h, J, pairs, dtau, U, hs, z, seed=seed, chain=c)
              for c, (hs, z) in enumerate(cfg)]
    for sweep in range(n_sweeps):
        st = ens.sweep(1)
        obs, sg, nm = ens.measure(reset=True)
        fields, _ = ens.get_fields()
        acc = 0
        for c in range(n_ch):
            kin_o, s_o, m2_o, a = chains[c].sweep()
            acc += a
            assert np.array_equal(fields[c][:, :N], chains[c].hs.reshape(L, N)), (sweep, c)
            assert np.array_equal(fields[c][:, N:], chains[c].ising.reshape(L, nb)), (sweep, c)
            _, _, _, P = ens.greens(c)
            assert abs(P - complex(chains[c].phase[0], chains[c].phase[1])) < 1e-9
            assert nm[c] == 1 and sg[c] == s_o
            assert abs(obs[c, 0] - kin_o) < 1e-8 * max(1.0, abs(kin_o))
            assert abs(obs[c, 4] - m2_o) < 1e-8 * max(1.0, abs(m2_o))
        assert st["accepted"] == acc and st["proposals"] == n_ch * 2 * L * (N + nb)
        assert 0 < acc < st["proposals"]
    ens.close()


def test_bond_model_rejects_bad_bonds(dq):
    K = W.chain_lattice(3)
    for kw in (dict(bonds=[(0, 0)], h=1.0), dict(bonds=[(0, 3)], h=1.0), dict(bonds=[(0, 1)], h=0.0),
               dict(bonds=[(0, 1)], h=1.0, pairs=[(0, 0)]), dict(bonds=[], pairs=[(0, 1)])):
        m = dq.Su2Model(K, U=2.0, dtau=0.1, L=4, n_wrap=2, xi=0.5, **kw)
        with pytest.raises(dq.DqmcError) as e:
            dq.Su2Ensemble([m], [0])
        assert e.value.status == dq.DQMC_EINVAL, kw
    m = dq.Su2Model(K, U=2.0, dtau=0.1, L=4, n_wrap=2, bonds=[(0, 1)], xi=0.5, h=1.0)
    bad = np.ones((4, 4), dtype=np.int8)
    bad[2, 3] = 2                      # a bond spin must be +-1
    with pytest.raises(dq.DqmcError) as e:
        dq.Su2Ensemble([m], [0], fields=[bad])
    assert e.value.status == dq.DQMC_EINVAL


# ------------------------------------------------- the samplers against ED
@pytest.mark.parametrize("mu", [0.0, 0.4])
def test_su2_sampler_matches_trotter_energy(dq, orc, mu):
    """256 GPU chains of the SU(2) decoupling on a dimer, reweighted by
    sign P / Re P (Sec. 2.2): the energy at tau = 0 agrees with the Fock-space
    trace of the Trotter product within 4 sigma (spread over the chains), at and
    away from half filling."""
    from paper_1704_00131_gb300 import analysis as A

    from .fock_ed import Fock, su2_trotter
    K, U, dtau, L = W.chain_lattice(2, t=1.0, mu=mu), 4.0, 0.25, 4
    eta = {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)}
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}
    _, Ef = su2_trotter(Fock(2), K, U, dtau, L, eta, gam)
    n_ch, burn, n = 256, 40, 300
    m = dq.Su2Model(K, U=U, dtau=dtau, L=L, n_wrap=2)
    ens = dq.Su2Ensemble([m], [0] * n_ch, seed=31 + int(10 * mu), measure=True, meas_first=0, meas_last=0)
    ens.sweep(burn)
    ens.measure(reset=True)
    st = ens.sweep(n)
    obs, sg, nm = ens.measure()
    ens.close()
    assert (nm == n).all() and 0 < st["accepted"] < st["proposals"]
    mean_re, err_re = A.jackknife(obs[:, 3].real / n, sg / n)
    mean_im, err_im = A.jackknife(obs[:, 3].imag / n, sg / n)
    assert abs(mean_re - Ef.real) < 4 * err_re, (mean_re, err_re, Ef)
    assert abs(mean_im) < 4 * err_im + 1e-12
    # power of the test: the energy scale of the dimer is ~1 (the energy itself is
    # ~0 at half filling, so the bar on the error is absolute)
    assert err_re < 0.1


@pytest.mark.parametrize("mu", [0.0, 0.4])
def test_bond_model_sampler_matches_trotter_product(dq, orc, mu):
    """256 GPU chains of the Hubbard-Ising model on a three-site chain with two
    bonds: the reweighted Kin and the bond spins' (sum_b s_b)^2 / n_bonds at
    tau = 0 agree with the trace of the Trotter product on Fock (x) Ising space
    within 4 sigma."""
    from paper_1704_00131_gb300 import analysis as A

    from .fock_ed import Fock, hubbard_ising_trotter
    K, U, dtau, L = W.chain_lattice(3, t=1.0, mu=mu), 2.0, 0.25, 4
    bonds, pairs = [(0, 1), (1, 2)], [(0, 1)]
    xi, h, J = 0.7, 0.8, 0.4
    eta = {l: orc.field_coupling(2, 1.0, 2.0, l) for l in (-2, -1, 1, 2)}
    gam = {l: orc.field_gamma(2, l) for l in (-2, -1, 1, 2)}
    _, kin_ref, m2_ref = hubbard_ising_trotter(Fock(3), K, U, dtau, L, eta, gam, bonds, xi, h, J, pairs,
                                               with_m2=True)
    n_ch, burn, n = 256, 40, 300
    m = dq.Su2Model(K, U=U, dtau=dtau, L=L, n_wrap=2, bonds=bonds, xi=xi, h=h, J=J, pairs=pairs)
    ens = dq.Su2Ensemble([m], [0] * n_ch, seed=57 + int(10 * mu), measure=True, meas_first=0, meas_last=0)
    ens.sweep(burn)
    ens.measure(reset=True)
    st = ens.sweep(n)
    obs, sg, nm = ens.measure()
    ens.close()
    assert (nm == n).all() and 0.05 < st["accepted"] / st["proposals"] < 0.95
    for q, ref in ((0, kin_ref.real), (4, m2_ref.real)):
        mean, err = A.jackknife(obs[:, q].real / n, sg / n)
        assert abs(mean - ref) < 4 * err, (q, mean, err, ref)
        assert err < 0.05 * abs(ref)


def test_su2_correlations_match_oracle(dq, orc):
    """Equal-time correlations per translation class (S^z S^z, n n, S^+ S^-,
    c^+ c) from the working G(0) of chains of two lattices in one context,
    against the oracle's correlations on its own stable G(0) for the same
    fields; after a sweep, against the oracle's formula applied to the GPU's
    working G."""
    ms = [dq.Su2Model(W.square_lattice(4, 4, t=1.0, mu=0.3), U=4.0, dtau=0.1, L=40, n_wrap=10),
          dq.Su2Model(W.square_lattice(3, 3, t=1.0), U=3.0, dtau=0.1, L=20, n_wrap=5)]
    cl = [W.translation_classes_square(4, 4), W.translation_classes_square(3, 3)]
    chain_model = [0, 1, 0]
    rng = np.random.default_rng(8)
    fields = [rng.choice([-2, -1, 1, 2], size=(ms[m].L, ms[m].N)).astype(np.int8) for m in chain_model]
    ens = dq.Su2Ensemble(ms, chain_model, fields=fields, seed=3)
    out, P = ens.measure_corr([c[0] for c in cl], [c[1] for c in cl])
    for c, m in enumerate(chain_model):
        mm, (cls, ncls, _) = ms[m], cl[m]
        Go, _, _ = orc.su2_green_udv(mm.hopping, mm.dtau, mm.U, mm.n_wrap, fields[c], 0)
        ref = orc.su2_correlations(Go, cls, ncls)
        assert np.abs(out[c, :ncls] - ref).max() < 1e-9 * max(1.0, np.abs(ref).max()), c
        assert np.all(out[c, ncls:] == 0)
        _, _, _, Pc = ens.greens(c)
        assert P[c] == Pc
    ens.sweep(1)
    out, _ = ens.measure_corr([c[0] for c in cl], [c[1] for c in cl])
    for c, m in enumerate(chain_model):
        G, _, _, _ = ens.greens(c)
        ref = orc.su2_correlations(G, cl[m][0], cl[m][1])
        assert np.abs(out[c, :cl[m][1]] - ref).max() < 1e-12 * max(1.0, np.abs(ref).max()), c
    with pytest.raises(dq.DqmcError) as e:
        bad = cl[0][0].copy()
        bad[1] = cl[0][1]                   # class index out of range
        ens.measure_corr([bad, cl[1][0]], [cl[0][1], cl[1][1]])
    assert e.value.status == dq.DQMC_EINVAL
    ens.close()


@pytest.mark.parametrize("mu,L,nw", [(0.0, 20, 5), (0.3, 20, 5), (-0.4, 60, 10)])
def test_su2_displaced_greens_match_oracle(dq, orc, mu, L, nw):
    """G(tau,0) and G(0,tau) (Sec. 2.4) of fixed fields: wrapped slice by slice
    from the stable G(0) and recomputed from the UDV chains at every multiple of
    n_wrap, against the oracle's displaced functions from its own UDV chains at
    taus on and between the recompute points; the traces of measure_tau are
    sum_x G(tau,0)_xx; the ends reduce to G(beta,0) = 1 - G(0), G(0,beta) = -G(0)."""
    K = W.square_lattice(4, 4, t=1.0, mu=mu)
    dtau, U, n_ch = 0.1, 4.0, 2
    rng = np.random.default_rng(int(L + 10 * mu) + 7)
    fields = [rng.choice([-2, -1, 1, 2], size=(L, 16)).astype(np.int8) for _ in range(n_ch)]
    m = dq.Su2Model(K, U=U, dtau=dtau, L=L, n_wrap=nw)
    ens = dq.Su2Ensemble([m], [0] * n_ch, fields=fields, seed=5)
    taus = sorted({0, 1, nw - 1, nw, nw + 3, L // 2, L - 1, L})
    a, (pmean, pmax) = ens.measure_tau(L)
    assert a.shape == (n_ch, L + 1)
    assert pmax < 1e-8 and pmean <= pmax
    for c in range(n_ch):
        G0, _, _ = orc.su2_green_udv(K, dtau, U, nw, fields[c], 0)
        for tau in taus:
            Gt0, G0t = ens.greens_displaced(c, tau)
            Ot0, O0t = orc.su2_green_displaced(K, dtau, U, nw, fields[c], tau)
            assert np.abs(Gt0 - Ot0).max() < 1e-9, (c, tau)
            assert np.abs(G0t - O0t).max() < 1e-9, (c, tau)
            assert abs(a[c, tau] - np.trace(Gt0)) < 1e-12 * max(1.0, abs(a[c, tau])), (c, tau)
            if tau == L:
                assert np.abs(Gt0 - (np.eye(16) - G0)).max() < 1e-9
                assert np.abs(G0t + G0).max() < 1e-9
            if tau == 0:
                assert np.abs(Gt0 - G0).max() < 1e-10 and np.abs(G0t - (G0 - np.eye(16))).max() < 1e-10
    ens.close()


def test_su2_tau_measurement_leaves_the_chain(dq):
    """The tau measurement rebuilds the stored chain it borrows: the working
    G(0), the phase and the next sweeps' field trajectory equal those of an
    identical ensemble that was not measured."""
    m = dq.Su2Model(W.square_lattice(4, 4, t=1.0, mu=0.2), U=4.0, dtau=0.1, L=40, n_wrap=10)
    e1 = dq.Su2Ensemble([m], [0] * 3, seed=21)
    e2 = dq.Su2Ensemble([m], [0] * 3, seed=21)
    e1.sweep(1)
    e2.sweep(1)
    before = [e1.greens(c) for c in range(3)]
    e1.measure_tau(17)
    e1.greens_displaced(1, 23)
    for c in range(3):
        G, la, ar, P = e1.greens(c)
        assert np.array_equal(G, before[c][0]) and P == before[c][3]
    s1, s2 = e1.sweep(2), e2.sweep(2)
    f1, _ = e1.get_fields()
    f2, _ = e2.get_fields()
    assert np.array_equal(f1, f2) and s1["accepted"] == s2["accepted"]
    for c in range(3):
        assert np.abs(e1.greens(c)[0] - e2.greens(c)[0]).max() < 1e-10
    with pytest.raises(dq.DqmcError) as e:
        e1.measure_tau(41)
    assert e.value.status == dq.DQMC_EINVAL
    with pytest.raises(dq.DqmcError) as e:
        e1.greens_displaced(1, 41)
    assert e.value.status == dq.DQMC_EINVAL
    e1.close()
    e2.close()


def test_su2_paper_example_precision_tau(dq):
    """4 x 4, U = 4, beta = 10, n_wrap = 10 (the paper's SU(2) example): the
    Precision tau of the time-displaced measurement over the whole interval
    stays at the level the paper reports for its example (mean ~1e-14, max
    ~1e-11)."""
    m = dq.Su2Model(W.square_lattice(4, 4), U=4.0, dtau=0.1, L=100, n_wrap=10)
    ens = dq.Su2Ensemble([m], [0] * 8, seed=11)
    ens.sweep(3)
    a, (pmean, pmax) = ens.measure_tau(100)
    assert pmean < 1e-12 and pmax < 1e-8
    assert np.all(np.isfinite(a)) and np.all(np.abs(a[:, 50]) < np.abs(a[:, 0]))
    ens.close()


def test_bond_model_displaced_greens(dq, orc):
    """Bond model (two-site bond factors inside each slice): the ends of the
    displaced functions against the oracle's G(0) (G(beta,0) = 1 - G(0),
    G(0,beta) = -G(0)); at an interior tau between recompute points, the
    identity -G(tau,0) G(0,tau) = G(tau) (1 - G(tau)) with the oracle's
    equal-time G(tau); Precision tau at the FP64 level."""
    Lx, L, nw = 3, 15, 5
    T = W.square_lattice(Lx, Lx, t=1.0, mu=0.2)
    bonds = _square_bonds(Lx, Lx)[:4]
    rng = np.random.default_rng(41)
    hs = [rng.choice([-2, -1, 1, 2], size=(L, 9)).astype(np.int8) for _ in range(2)]
    ising = [rng.choice([-1, 1], size=(L, len(bonds))).astype(np.int8) for _ in range(2)]
    m = dq.Su2Model(T, U=3.0, dtau=0.1, L=L, n_wrap=nw, bonds=bonds, xi=0.5, h=1.0, J=0.0)
    ens = dq.Su2Ensemble([m], [0, 0], fields=[np.concatenate([hs[c], ising[c]], axis=1) for c in range(2)], seed=3)
    _, (pmean, pmax) = ens.measure_tau(L)
    assert pmax < 1e-9
    for c in range(2):
        G0, _, _ = orc.hubbard_ising_green_udv(T, bonds, 0.5, 0.1, 3.0, nw, hs[c], ising[c], 0)
        Gt0, G0t = ens.greens_displaced(c, L)
        assert np.abs(Gt0 - (np.eye(9) - G0)).max() < 1e-9
        assert np.abs(G0t + G0).max() < 1e-9
        for tau in (3, 7, 12):
            Gt, _, _ = orc.hubbard_ising_green_udv(T, bonds, 0.5, 0.1, 3.0, nw, hs[c], ising[c], tau)
            Gt0, G0t = ens.greens_displaced(c, tau)
            assert np.abs(-Gt0 @ G0t - Gt @ (np.eye(9) - Gt)).max() < 1e-9, (c, tau)
    ens.close()
