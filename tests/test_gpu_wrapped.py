"""Interior-slice parity of the wrapped Green function (Sec. 2.3).

Between stabilisations a sweep carries G(tau) by the wraps
G <- B_tau G B_tau^-1 in its working precision, and round-off grows with the
condition number of the product of the slices since the last stabilisation.
dqmc_greens_tau returns that wrapped G at any tau on the chain's current fields
(the sweep's arithmetic with every proposal rejected, i.e. on frozen fields).  It
is compared element by element with the FP64 oracle's stable G(tau) on the same
fields at the slices furthest from a stabilisation point (tau0 + n_wrap - 1),
for one chain of the hardest class of the 256-chain workload (12x12, beta = 8,
U = 6) and one of the lightest (8x8, beta = 4, U = 2), on the FP64 and the
float-pair paths.  At a stabilisation point (tau = tau0) no wrap has happened and
the returned G is the stable recompute itself.

Bars.  At U = 6 and n_wrap = 10 the product of ten slices is so badly
conditioned that the FP64 oracle's own stable G moves by delta =
max |G_oracle(n_wrap = 10) - G_oracle(n_wrap = 5)| (3e-8 on the 8x8, beta = 8
configuration here, 3e-10 on the 12x12 one, 1e-13 at U = 2): round-off of
unit size u is amplified by the condition number of ten slices, and every path
inherits that amplification with its own u.  With delta measured here from the
oracle alone, max |G_wrap - G_oracle| over the sampled slices must stay below
* FP64 path: max(1e-9, 100 delta);
* float-pair paths (u about 2^-44 for the float-pair products, 2^-48 storage):
  max(1e-6, 1000 delta) -- the reduced-precision target of 1e-6 wherever the
  FP64 stabilisation itself is good to 1e-9.
At a stabilisation point (tau = tau0, no wrap) the same bars apply to the stable
recompute.
"""
import numpy as np
import pytest

from paper_1704_00131_gb300 import workloads as W

pytestmark = pytest.mark.gpu

BAR = {"fp64": (1e-9, 100.0), "mixed": (1e-6, 1000.0), "mixed_tc": (1e-6, 1000.0)}


@pytest.fixture(scope="module")
def dq():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00131_gb300 import build_ext, dqmc
    build_ext.build()
    return dqmc


def _model(n, beta, U):
    return W.ModelSpec(W.square_lattice(n, n), U=U, dtau=0.1, L=int(round(beta / 0.1)), n_wrap=10)


CASES = {"square12x12_b8_U6": (12, 8.0, 6.0), "square8x8_b8_U6": (8, 8.0, 6.0), "square8x8_b4_U2": (8, 4.0, 2.0)}


@pytest.fixture(scope="module")
def oracle_greens(orc):
    out = {}
    for name, (n, beta, U) in CASES.items():
        m = _model(n, beta, U)
        f = W.random_fields(1, m.L, m.n_vertices, seed=8)
        om = orc.Model(m.hopping, m.vertex_site, m.vertex_sign, m.U, m.dtau, m.L, m.n_wrap, m.field_type)
        om5 = orc.Model(m.hopping, m.vertex_site, m.vertex_sign, m.U, m.dtau, m.L, 5, m.field_type)
        taus = [0, 9, m.L // 2 - 1, m.L - 1]
        ref = {(t, s): orc.green_udv(om, f, s, t)[0] for t in taus for s in (0, 1)}
        delta = max(float(np.abs(ref[(t, s)] - orc.green_udv(om5, f, s, t)[0]).max()) for t in (0, m.L // 2 - 1)
                    for s in (0, 1) if t % 5 == 0)
        out[name] = (m, f, ref, delta)
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_tc"])
@pytest.mark.parametrize("case", list(CASES))
def test_wrapped_green_at_interior_slices(dq, oracle_greens, case, precision):
    m, f, ref, delta = oracle_greens[case]
    floor, factor = BAR[precision]
    bar = max(floor, factor * delta)
    ens = dq.Ensemble([m], [0], fields=[f], precision=precision, delay_k=16)
    worst = 0.0
    for (t, s), Go in ref.items():
        Gw = ens.greens_tau(0, s, t)
        worst = max(worst, float(np.abs(Gw - Go).max()))
    assert worst < bar, (case, precision, worst, delta)
    # the fields and the working G(0) are left as they were
    fa, _ = ens.get_fields()
    assert np.array_equal(fa[0], f)
    ens.close()


def test_wrapped_green_rejects_bad_tau(dq):
    m = _model(4, 2.0, 4.0)
    ens = dq.Ensemble([m], [0], precision="fp64")
    with pytest.raises(dq.DqmcError) as e:
        ens.greens_tau(0, 0, m.L + 1)
    assert e.value.status == dq.DQMC_EINVAL
    ens.close()
