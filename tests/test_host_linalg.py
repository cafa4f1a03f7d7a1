"""The library's host-side set-up of e^{-dtau K} (row a1, Sec. 3.1 Op_set) on the CPU.

dqmc_init and dqmc_su2_init diagonalise each model's hopping matrix once on the
host (Jacobi rotations, csrc/dqmc_linalg_host.h) and build e^{-+dtau K} from the
eigenpairs.  On a GPU-less machine dqmc_init stops before that step, so these
tests compile the header alone with g++ into a small shim and check it against
LAPACK (numpy.linalg.eigh) and scipy's Pade exponential on the lattices of the
benchmark workloads: square 4x4, 8x8, 12x12, 20x20 with t' and mu, honeycomb
6x6, a ragged open chain, and a random symmetric matrix with clustered
eigenvalues.  Square lattices have heavily degenerate spectra, which a Jacobi
method has to resolve into an orthonormal eigenbasis.
"""
import os
import subprocess

import numpy as np
import pytest

from paper_1704_00131_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1704_00131_gb300", "csrc")

SHIM = r"""
#include "dqmc_linalg_host.h"
#include <cstring>
extern "C" void shim_eigen(int n, const double* A, double* w, double* V) {
  std::vector<double> a(A, A + (size_t)n * n), ww, vv;
  dqmc::host::symmetric_eigen(n, a, ww, vv);
  std::memcpy(w, ww.data(), sizeof(double) * n);
  std::memcpy(V, vv.data(), sizeof(double) * n * n);
}
extern "C" void shim_expm(int n, const double* w, const double* V, double t, double* E) {
  std::vector<double> ww(w, w + n), vv(V, V + (size_t)n * n);
  std::vector<double> e = dqmc::host::expm_symmetric(n, ww, vv, t);
  std::memcpy(E, e.data(), sizeof(double) * n * n);
}
"""


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    import ctypes
    d = tmp_path_factory.mktemp("linalg_host")
    src = d / "shim.cpp"
    src.write_text(SHIM)
    so = d / "libshim.so"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", CSRC, "-o", str(so), str(src)])
    lib = ctypes.CDLL(str(so))
    vp = ctypes.c_void_p
    lib.shim_eigen.argtypes = [ctypes.c_int, vp, vp, vp]
    lib.shim_expm.argtypes = [ctypes.c_int, vp, vp, ctypes.c_double, vp]

    def eigen(A):
        A = np.ascontiguousarray(A, dtype=np.float64)
        n = A.shape[0]
        w, V = np.zeros(n), np.zeros((n, n))
        lib.shim_eigen(n, A.ctypes.data, w.ctypes.data, V.ctypes.data)
        return w, V

    def expm(w, V, t):
        w = np.ascontiguousarray(w, dtype=np.float64)
        V = np.ascontiguousarray(V, dtype=np.float64)
        n = w.shape[0]
        E = np.zeros((n, n))
        lib.shim_expm(n, w.ctypes.data, V.ctypes.data, float(t), E.ctypes.data)
        return E

    return eigen, expm


def _clustered(n=40, seed=5):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    w = np.repeat(rng.standard_normal(n // 4), 4) + 1e-9 * rng.standard_normal(n)
    A = (Q * w) @ Q.T
    return 0.5 * (A + A.T)


LATTICES = {
    "square4x4": lambda: W.square_lattice(4, 4),
    "square8x8": lambda: W.square_lattice(8, 8),
    "square12x12": lambda: W.square_lattice(12, 12),
    "square20x20_tp_mu": lambda: W.square_lattice(20, 20, 1.0, -0.2, -0.5),
    "honeycomb6x6": lambda: W.honeycomb_lattice(6, 6),
    "chain13_open": lambda: W.chain_lattice(13, t=1.0, mu=0.3, periodic=False),
    "clustered40": _clustered,
}


@pytest.mark.parametrize("name", list(LATTICES))
def test_host_eigendecomposition_and_propagator(shim, name):
    eigen, expm = shim
    from scipy.linalg import expm as scipy_expm
    K = LATTICES[name]()
    n = K.shape[0]
    scale = max(1.0, np.abs(K).max())
    w, V = eigen(K)
    assert np.abs(np.sort(w) - np.linalg.eigvalsh(K)).max() < 1e-13 * scale * np.sqrt(n)
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13 * np.sqrt(n)
    assert np.abs((V * w) @ V.T - K).max() < 1e-13 * scale * np.sqrt(n)
    for dtau in (0.1, 0.05):
        E = expm(w, V, -dtau)
        Einv = expm(w, V, +dtau)
        ref = scipy_expm(-dtau * K)
        assert np.abs(E - ref).max() < 1e-14 * np.sqrt(n) * max(1.0, np.abs(ref).max())
        assert np.abs(E @ Einv - np.eye(n)).max() < 1e-13 * np.sqrt(n)
        assert np.abs(E - E.T).max() < 1e-15 * np.sqrt(n)
