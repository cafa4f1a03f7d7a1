"""The allocation-free entry point dqmc_green_fresh_noalloc.

Some callers cannot allocate device memory where they need a Green function:
code running under an allocator that owns every device allocation, or a context
that must not call cudaMalloc.  For them the library offers one entry point that
takes only caller-owned device buffers and keeps its scratch in a fixed device
array of the library.  These tests call it through the C ABI and compare it with
the FP64 oracle's G(0) and log|det| on the same fields and with
dqmc_greens(fresh=1), which computes the same G(0) with the context's own
allocations, on two calls in a row with different fields (the scratch array keeps
the previous call's contents, which must not leak into the next result), for two
flavors of Ising fields at the size limit and for one flavor of four-valued
fields on a smaller lattice (a leading dimension other than the limit's).
This file is collected last so that a failure here stops a run only after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_1704_00131_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def noalloc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_00131_gb300 import build_ext, dqmc
    build_ext.build()
    lib = dqmc.load()
    fn = lib.dqmc_green_fresh_noalloc
    vp, i32, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double
    fn.argtypes = [i32, i32, vp, i32, vp, vp, d, i32, d, i32, i32, vp, vp, vp, vp, vp]
    fn.restype = ctypes.c_int
    return dqmc, fn


def _exp_minus_dtau_K(K: np.ndarray, dtau: float) -> np.ndarray:
    w, V = np.linalg.eigh(K)
    return (V * np.exp(-dtau * w)) @ V.T


@pytest.mark.parametrize("case", ["square8x8_ising_2fl", "square6x6_hs4_1fl"])
def test_noalloc_matches_oracle_and_fresh_green_on_two_calls(noalloc, orc, case):
    import torch
    dqmc, fn = noalloc
    if case == "square8x8_ising_2fl":
        m = W.ModelSpec(W.square_lattice(8, 8), U=4.0, dtau=0.1, L=40, n_wrap=10)  # N = 64, the limit
        nfl = 2
    else:
        K = W.square_lattice(6, 6, 1.0, -0.2, -0.3)
        m = W.ModelSpec(K, U=3.0, dtau=0.1, L=30, n_wrap=5, field_type=2)
        m = W.ModelSpec(m.hopping[:1], U=m.U, dtau=m.dtau, L=m.L, n_wrap=m.n_wrap, field_type=2,
                        vertex_site=m.vertex_site, vertex_sign=m.vertex_sign[:1])
        nfl = 1
    N, MV = m.N, m.n_vertices
    om = orc.Model(m.hopping, m.vertex_site, m.vertex_sign, m.U, m.dtau, m.L, m.n_wrap, m.field_type)
    dev = torch.device("cuda", 0)
    E = torch.from_numpy(np.stack([_exp_minus_dtau_K(m.hopping[s], m.dtau) for s in range(nfl)])).to(dev)
    site = torch.from_numpy(m.vertex_site).to(dev)
    sign = torch.from_numpy(m.vertex_sign).to(dev)
    G = torch.empty((nfl, N, N), dtype=torch.float64, device=dev)
    ld = torch.empty(nfl, dtype=torch.float64, device=dev)
    sg = torch.empty(nfl, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((101, 202)):
        f = W.random_fields(m.field_type, m.L, MV, seed=seed)
        fd = torch.from_numpy(f).to(dev)
        st = fn(N, nfl, E.data_ptr(), MV, site.data_ptr(), sign.data_ptr(), m.U, m.field_type, m.dtau, m.L,
                m.n_wrap, fd.data_ptr(), G.data_ptr(), ld.data_ptr(), sg.data_ptr(), stream.cuda_stream)
        assert st == dqmc.DQMC_OK, f"call {call}: status {st}"
        torch.cuda.synchronize()
        ens = dqmc.Ensemble([m], [0], fields=[f], precision="fp64")
        for s in range(nfl):
            Gs = G[s].cpu().numpy()
            Go, ldo, sgo = orc.green_udv(om, f, s, 0)
            assert np.abs(Gs - Go).max() < 1e-10, f"call {call}, flavor {s}: oracle"
            assert float(ld[s]) == pytest.approx(ldo, rel=1e-10, abs=1e-10)
            assert int(sg[s]) == sgo
            Gref, ldref, sgref = ens.greens(0, s, fresh=True)
            assert np.abs(Gs - Gref).max() < 1e-10, f"call {call}, flavor {s}"
            assert float(ld[s]) == pytest.approx(ldref, rel=1e-10, abs=1e-10)
            assert int(sg[s]) == sgref
        ens.close()


def test_noalloc_reports_invalid_vertex_sites(noalloc):
    """The vertex sites are device data the host cannot check: the kernel checks
    them (distinct, in [0, N)) before using them and answers sign 0 and a G of NaNs."""
    import torch
    dqmc, fn = noalloc
    m = W.ModelSpec(W.square_lattice(4, 4), U=4.0, dtau=0.1, L=10, n_wrap=5)
    N, MV = m.N, m.n_vertices
    dev = torch.device("cuda", 0)
    E = torch.from_numpy(np.stack([_exp_minus_dtau_K(m.hopping[s], m.dtau) for s in range(2)])).to(dev)
    sign = torch.from_numpy(m.vertex_sign).to(dev)
    fd = torch.from_numpy(W.random_fields(1, m.L, MV, seed=3)).to(dev)
    stream = torch.cuda.current_stream()
    for bad in ([N] + list(range(1, N)), [0, 0] + list(range(2, N))):   # one past the end; a duplicate
        site = torch.tensor(bad, dtype=torch.int32, device=dev)
        G = torch.zeros((2, N, N), dtype=torch.float64, device=dev)
        ld = torch.ones(2, dtype=torch.float64, device=dev)
        sg = torch.ones(2, dtype=torch.int32, device=dev)
        st = fn(N, 2, E.data_ptr(), MV, site.data_ptr(), sign.data_ptr(), m.U, 1, m.dtau, m.L, m.n_wrap,
                fd.data_ptr(), G.data_ptr(), ld.data_ptr(), sg.data_ptr(), stream.cuda_stream)
        assert st == dqmc.DQMC_OK
        torch.cuda.synchronize()
        assert sg.cpu().tolist() == [0, 0] and ld.cpu().tolist() == [0.0, 0.0]
        assert bool(torch.isnan(G).all())


def test_noalloc_rejects_sizes_beyond_the_limit(noalloc):
    import torch
    dqmc, fn = noalloc
    N = 65
    dev = torch.device("cuda", 0)
    E = torch.zeros((2, N, N), dtype=torch.float64, device=dev)
    site = torch.arange(N, dtype=torch.int32, device=dev)
    sign = torch.ones((2, N), dtype=torch.float64, device=dev)
    f = torch.ones((10, N), dtype=torch.int8, device=dev)
    G = torch.empty((2, N, N), dtype=torch.float64, device=dev)
    st = fn(N, 2, E.data_ptr(), N, site.data_ptr(), sign.data_ptr(), 4.0, 1, 0.1, 10, 10, f.data_ptr(),
            G.data_ptr(), None, None, None)
    assert st == dqmc.DQMC_EINVAL
