"""GPU parity of the time-displaced measurement (dqmc_measure_tau) against the oracle.

The GPU wraps G(tau,0), G(0,tau), G(tau,tau) slice by slice between the
stabilisation points; the oracle recomputes every one from scratch through the
UDV chains.  Both are FP64, so each Green-function entry agrees to the 1e-10
of the FP64 paths; the sums a (N terms), p (N terms) and c (N^2 products of
O(1) entries) are compared at N * 1e-10, N * 1e-10 and 2 N^2 * 1e-10.
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


def omodel(orc, m):
    return orc.Model(m.hopping, m.vertex_site, m.vertex_sign, m.U, m.dtau, m.L, m.n_wrap, m.field_type)


def check_chain(orc, m, fields, obs_c, sign_c, n_tau, ph):
    om = omodel(orc, m)
    ntc = min(n_tau, m.L)
    ref, sg = orc.tau_observables(om, fields, ntc, ph)
    N = m.N
    tol = np.array([N * 1e-10, 2 * N * N * 1e-10, N * 1e-10])
    d = np.abs(obs_c[:ntc + 1] - ref)
    assert (d <= tol).all(), f"max diff per quantity {d.max(axis=(0, 1))}, tolerance {tol}"
    assert np.all(obs_c[ntc + 1:] == 0.0)
    assert list(sign_c) == list(sg)


@pytest.mark.parametrize("ft", [1, 2])
def test_tau_measure_single_chain(dq, orc, ft):
    m = W.ModelSpec(W.square_lattice(4, 4, tp=-0.1, mu=-0.3), U=4.0, dtau=0.1, L=20, n_wrap=5, field_type=ft)
    f = W.random_fields(ft, m.L, m.n_vertices, seed=17)
    ens = dq.Ensemble([m], [0], fields=[f], precision="fp64")
    ph = W.sublattice_signs_square(4, 4)
    obs, sg, prec = ens.measure_tau(m.L, [ph])
    check_chain(orc, m, f, obs[0], sg[0], m.L, ph)
    assert 0.0 <= prec[0] < 1e-11 and prec[1] < 1e-9
    # partial window
    obs2, _, _ = ens.measure_tau(7, [ph])
    assert np.abs(obs2[0] - obs[0, :8]).max() < 1e-12
    ens.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tau_measure_batch_leaves_the_chains_alone(dq, orc, precision):
    """Uneven chains after a sweep: every chain matches the oracle on its current
    fields, and a twin ensemble that is not measured continues bit for bit alike."""
    models = [W.ModelSpec(W.square_lattice(4, 4), U=4.0, dtau=0.1, L=20, n_wrap=10),
              W.ModelSpec(W.honeycomb_lattice(3, 3), U=3.0, dtau=0.1, L=10, n_wrap=5),
              W.ModelSpec(W.chain_lattice(13, mu=0.2, periodic=True), U=2.0, dtau=0.125, L=16, n_wrap=4,
                          field_type=2)]
    cm = [0, 1, 2, 0]
    phases = [W.sublattice_signs_square(4, 4), W.sublattice_signs_honeycomb(3, 3),
              np.cos(np.pi * np.arange(13) / 6.5)]
    a = dq.Ensemble(models, cm, precision=precision, delay_k=8, seed=5)
    b = dq.Ensemble(models, cm, precision=precision, delay_k=8, seed=5)
    a.sweep(1)
    b.sweep(1)
    fa, _ = a.get_fields()
    G_before = [a.greens(c, s)[0] for c in range(len(cm)) for s in (0, 1)]
    n_tau = 20
    obs, sg, prec = a.measure_tau(n_tau, phases)
    for c in range(len(cm)):
        mi = cm[c]
        check_chain(orc, models[mi], fa[c], obs[c], sg[c], n_tau, phases[mi])
    assert prec[1] < 1e-8
    G_after = [a.greens(c, s)[0] for c in range(len(cm)) for s in (0, 1)]
    assert all(np.array_equal(x, y) for x, y in zip(G_before, G_after))
    a.sweep(2)
    b.sweep(2)
    fa2, ca = a.get_fields()
    fb2, cb = b.get_fields()
    assert ca == cb and all(np.array_equal(x, y) for x, y in zip(fa2, fb2))
    for c in range(len(cm)):
        for s in (0, 1):
            assert np.array_equal(a.greens(c, s)[0], b.greens(c, s)[0])
    a.close()
    b.close()


def test_tau_measure_spin_correlation_identity(dq):
    """tau = 0 of the S^z S^z sum equals the equal-time value from G(0):
    sum_xy ph_x ph_y <S^z_x S^z_y> with the same Wick rule at equal times."""
    m = W.ModelSpec(W.square_lattice(6, 6), U=4.0, dtau=0.1, L=20, n_wrap=10)
    ens = dq.Ensemble([m], [0], precision="fp64", seed=3)
    ens.sweep(1)
    ph = W.sublattice_signs_square(6, 6)
    obs, _, _ = ens.measure_tau(4, [ph])
    szz = dq.szz_tau(obs)[0]
    G = [ens.greens(0, s, fresh=True)[0] for s in (0, 1)]
    n = [1.0 - np.diag(g) for g in G]
    mz = np.sum(ph * (n[0] - n[1]))
    conn = sum(np.einsum("x,y,yx,xy->", ph, ph, np.eye(36) - g, g) for g in G)
    assert szz[0] == pytest.approx((mz * mz + conn) / 4.0, rel=1e-10, abs=1e-10)
    ens.close()


def test_tau_measure_invalid_arguments(dq):
    m = W.ModelSpec(W.square_lattice(4, 4), U=4.0, dtau=0.1, L=20, n_wrap=10)
    ens = dq.Ensemble([m], [0], precision="fp64", seed=1)
    for bad in (-1, 21):
        with pytest.raises(dq.DqmcError) as e:
            ens.measure_tau(bad)
        assert e.value.status == dq.DQMC_EINVAL
    with pytest.raises(dq.DqmcError):
        ens.measure_tau(4, [np.ones(3)])
    with pytest.raises(dq.DqmcError) as e:
        ens.measure_tau(4, [np.full(16, np.nan)])
    assert e.value.status == dq.DQMC_EINVAL
    ens.close()


# ------------------------------------------- class-resolved correlation functions
def test_tau_correlations_per_pair_against_the_oracle(dq, orc):
    """One class per ordered pair (x, y) on a lattice without inversion symmetry
    (3x3 torus with t', a site potential and one modified bond): the pair's
    sum_s G^s(tau,0)_xy, <S^z_x(tau) S^z_y(0)> and <n_x(tau) n_y(0)> against the
    oracle's, which recomputes every Green function from scratch, for every tau
    (wrapped slices and stabilisation points, n_wrap = 5).  A transposed or
    mis-signed entry of G(tau,0) or G(0,tau) fails here: no symmetry hides it."""
    K = W.square_lattice(3, 3, 1.0, -0.2, 0.1)
    K[0, 0] -= 0.3
    K[1, 5] = K[5, 1] = -0.35
    m = W.ModelSpec(K, U=4.0, dtau=0.1, L=20, n_wrap=5)
    N = m.N
    f = W.random_fields(1, m.L, N, seed=31)
    ens = dq.Ensemble([m], [0], fields=[f], precision="fp64")
    cls = np.arange(N * N, dtype=np.int32)
    out, sg = ens.measure_tau_corr(m.L, [cls], [N * N])
    ref = orc.tau_correlations(omodel(orc, m), f, m.L, cls, N * N)
    assert out.shape == (1, m.L + 1, N * N, 3)
    assert np.abs(out[0] - ref).max() < 1e-10
    _, sgo = orc.tau_observables(omodel(orc, m), f, 0)
    assert sg[0] == sgo[0] * sgo[1]
    ens.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_tau_correlations_batch_translation_classes(dq, orc, precision):
    """Uneven chains after a sweep, translation (displacement) classes of their
    own lattices: each chain's class sums against the oracle on its current fields;
    rows beyond the chain's L and classes beyond its model's count are 0."""
    models = [W.ModelSpec(W.square_lattice(4, 4, tp=-0.1), U=4.0, dtau=0.1, L=20, n_wrap=10),
              W.ModelSpec(W.honeycomb_lattice(3, 3), U=3.0, dtau=0.1, L=10, n_wrap=5),
              W.ModelSpec(W.chain_lattice(7, mu=0.2, periodic=True), U=2.0, dtau=0.125, L=16, n_wrap=4,
                          field_type=2)]
    chain_cls = np.array([[(j - i) % 7 for j in range(7)] for i in range(7)], dtype=np.int32).ravel()
    classes = [W.translation_classes_square(4, 4)[:2], W.translation_classes_honeycomb(3, 3)[:2], (chain_cls, 7)]
    cm = [0, 1, 2, 0]
    ens = dq.Ensemble(models, cm, precision=precision, delay_k=8, seed=9)
    ens.sweep(1)
    fa, _ = ens.get_fields()
    n_tau = 20
    out, sg = ens.measure_tau_corr(n_tau, [c for c, _ in classes], [n for _, n in classes])
    max_cls = max(n for _, n in classes)
    assert out.shape == (len(cm), n_tau + 1, max_cls, 3)
    for c, mi in enumerate(cm):
        m = models[mi]
        cl, nc = classes[mi]
        ntc = min(n_tau, m.L)
        ref = orc.tau_correlations(omodel(orc, m), fa[c], ntc, cl, nc)
        # each class sums N pairs of products of O(1) entries
        assert np.abs(out[c, :ntc + 1, :nc] - ref).max() < 2 * m.N * 1e-10, c
        assert np.all(out[c, ntc + 1:] == 0.0) and np.all(out[c, :, nc:] == 0.0)
    ens.close()


def test_tau_correlations_invalid_arguments(dq):
    m = W.ModelSpec(W.square_lattice(2, 2), U=4.0, dtau=0.1, L=10, n_wrap=5)
    ens = dq.Ensemble([m], [0], precision="fp64")
    cls = np.zeros(16, dtype=np.int32)
    with pytest.raises(dq.DqmcError) as e:
        ens.measure_tau_corr(11, [cls], [1])
    assert e.value.status == dq.DQMC_EINVAL
    cls[3] = 2
    with pytest.raises(dq.DqmcError) as e:
        ens.measure_tau_corr(4, [cls], [2])
    assert e.value.status == dq.DQMC_EINVAL
    ens.close()
