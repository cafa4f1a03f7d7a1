"""GPU parity of the equal-time correlation functions (dqmc_measure_corr).

Two references: the oracle's sums on the GPU's own working G (the kernel's
arithmetic, to rounding), and the oracle's sums on the oracle's G(0) for the same
fields.  For the second, every G entry agrees to the path's G tolerance g (1e-10
FP64, 1e-7 float pairs, 1e-6 FP32) and each pair term is a product of O(1)
entries, so a class of P pairs agrees to 8 P g.
"""
import numpy as np
import pytest

from paper_1704_00131_gb300 import workloads as W

pytestmark = pytest.mark.gpu

G_TOL = {"fp64": 1e-10, "mixed": 1e-7, "fp32": 1e-6}


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


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
def test_correlations_match_oracle(dq, orc, precision):
    models = [W.ModelSpec(W.square_lattice(4, 4, tp=-0.1, mu=-0.2), U=4.0, dtau=0.1, L=20, n_wrap=10),
              W.ModelSpec(W.honeycomb_lattice(3, 3), U=3.0, dtau=0.1, L=10, n_wrap=5, field_type=2)]
    classes = [W.translation_classes_square(4, 4), W.translation_classes_honeycomb(3, 3)]
    cm = [0, 1, 0]
    ens = dq.Ensemble(models, cm, precision=precision, delay_k=8, seed=9)
    ens.sweep(2)
    out, sg = ens.measure_corr([c[0] for c in classes], [c[1] for c in classes])
    fields, _ = ens.get_fields()
    nmax = max(c[1] for c in classes)
    assert out.shape == (3, nmax, 4)
    for c, mi in enumerate(cm):
        m, (cls, n, _) = models[mi], classes[mi]
        Gg = np.stack([ens.greens(c, s)[0] for s in (0, 1)])
        own = orc.correlations(Gg, cls, n)
        assert np.abs(out[c, :n] - own).max() < 1e-12
        assert np.all(out[c, n:] == 0.0)
        Go, sgo = [], 1
        for s in (0, 1):
            g, _, sign = orc.green_udv(omodel(orc, m), fields[c], s, 0)
            Go.append(g)
            sgo *= sign
        ref = orc.correlations(np.stack(Go), cls, n)
        pairs = np.bincount(cls, minlength=n)[:, None]
        assert (np.abs(out[c, :n] - ref) <= 8 * pairs * G_TOL[precision]).all()
        assert sg[c] == sgo
    ens.close()


def test_correlations_reject_bad_classes(dq):
    m = W.ModelSpec(W.square_lattice(4, 4), U=4.0, dtau=0.1, L=20, n_wrap=10)
    ens = dq.Ensemble([m], [0], precision="fp64", seed=1)
    cls, n, _ = W.translation_classes_square(4, 4)
    bad = cls.copy()
    bad[5] = n
    with pytest.raises(dq.DqmcError) as e:
        ens.measure_corr([bad], [n])
    assert e.value.status == dq.DQMC_EINVAL
    with pytest.raises(dq.DqmcError):
        ens.measure_corr([cls[:-1]], [n])
    out, _ = ens.measure_corr([np.full(256, -1, dtype=np.int32)], [1])
    assert np.all(out == 0.0)
    ens.close()
