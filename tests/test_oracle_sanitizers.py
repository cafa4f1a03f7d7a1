"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (CPU).

The oracle is plain C with hand-written loops over row-major arrays; an index
off by one would not necessarily change a pinned value.  Here the oracle is
built with -fsanitize=address,undefined into a temporary directory and every
oracle pin runs against that build (loaded through DQMC_ORACLE_LIB, the
sanitizer runtimes preloaded into the Python process): an out-of-bounds
access, a use after free or undefined behaviour aborts the run.  A control
first shows that the harness does catch a planted heap overflow in a separate
two-line library, so a clean run means a clean oracle and not an inactive
sanitizer.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_su2_pins.py", "tests/test_oracle_tau_pins.py",
        "tests/test_oracle_tau_corr_pins.py", "tests/test_oracle_corr_pins.py",
        "tests/test_oracle_bond_ising_pins.py", "tests/test_oracle_svd_pins.py"]
FLAGS = ["-O1", "-g", "-std=c99", "-fPIC", "-shared", "-fsanitize=address,undefined",
         "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]


def _runtime(name):
    p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


@pytest.fixture(scope="module")
def sanitized_env():
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not (asan and ubsan):
        pytest.skip("gcc has no sanitizer runtimes here")
    return dict(os.environ, LD_PRELOAD=f"{asan}:{ubsan}", ASAN_OPTIONS="detect_leaks=0",
                UBSAN_OPTIONS="print_stacktrace=1")


def test_harness_catches_a_heap_overflow(tmp_path, sanitized_env):
    src = tmp_path / "overflow.c"
    src.write_text("#include <stdlib.h>\n"
                   "double read_past_end(int n) { double* a = (double*)calloc(n, sizeof(double));\n"
                   "  double x = a[n]; free(a); return x; }\n")
    so = tmp_path / "liboverflow.so"
    subprocess.check_call(["gcc", *FLAGS, "-o", str(so), str(src)])
    code = ("import ctypes; f = ctypes.CDLL(%r).read_past_end; f.restype = ctypes.c_double; f(8)" % str(so))
    r = subprocess.run([sys.executable, "-c", code], env=sanitized_env, capture_output=True, text=True, timeout=300)
    # UBSan's object-size check or ASan's shadow memory, whichever sees it first
    assert r.returncode != 0 and ("heap-buffer-overflow" in r.stderr or "runtime error" in r.stderr), r.stderr[-2000:]


def test_oracle_pins_clean_under_sanitizers(tmp_path, sanitized_env):
    so = tmp_path / "liboracle.so"
    subprocess.check_call(["gcc", *FLAGS, "-o", str(so), os.path.join(ROOT, "oracle", "dqmc_oracle.c"), "-lm"])
    env = dict(sanitized_env, DQMC_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", *PINS, "-q", "-m", "not gpu", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    report = r.stdout[-3000:] + r.stderr[-3000:]
    assert r.returncode == 0, report
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, report


def test_library_host_linalg_clean_under_sanitizers(tmp_path, sanitized_env):
    """The library's host set-up of e^{-+dtau K} (the Jacobi eigendecomposition of
    csrc/dqmc_linalg_host.h, run inside dqmc_init) under the same sanitizers, on
    the square 8 x 8, the honeycomb 3 x 3 and a one-site lattice."""
    from tests.test_host_linalg import SHIM
    src = tmp_path / "shim.cpp"
    src.write_text(SHIM)
    so = tmp_path / "libshim.so"
    flags = [f for f in FLAGS if f != "-std=c99"] + ["-std=c++17"]
    subprocess.check_call(["g++", *flags, "-I", os.path.join(ROOT, "paper_1704_00131_gb300", "csrc"), "-o", str(so),
                           str(src)])
    code = f"""
import ctypes, sys
import numpy as np
sys.path.insert(0, {ROOT!r})
from paper_1704_00131_gb300 import workloads as W
lib = ctypes.CDLL({str(so)!r})
for K in (W.square_lattice(8, 8), W.honeycomb_lattice(3, 3), np.array([[0.3]])):
    K = np.ascontiguousarray(K, dtype=np.float64)
    n = K.shape[0]
    w, V, E = np.zeros(n), np.zeros((n, n)), np.zeros((n, n))
    lib.shim_eigen(n, K.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p), V.ctypes.data_as(ctypes.c_void_p))
    lib.shim_expm(n, w.ctypes.data_as(ctypes.c_void_p), V.ctypes.data_as(ctypes.c_void_p), ctypes.c_double(-0.1),
                  E.ctypes.data_as(ctypes.c_void_p))
    assert np.abs((V * w) @ V.T - K).max() < 1e-12
"""
    r = subprocess.run([sys.executable, "-c", code], cwd=os.path.join(ROOT, "tests"), env=sanitized_env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "runtime error" not in r.stderr, r.stderr[-3000:]
