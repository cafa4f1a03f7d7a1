"""Planted mistakes in the host analysis: each must fail a test of it.

The R -> K transform, the momentum grid and the jackknife of
paper_1704_00131_gb300/analysis.py are pinned by closed forms and plain
definitions in test_analysis_host.py (and the bin driver's tests).  Each case
plants one plausible mistake into a copy of the package's Python sources in a
temporary directory and runs those tests against the copy; they must fail.  The
unplanted copy must pass them.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = "paper_1704_00131_gb300"
TESTS = ["tests/test_analysis_host.py", "tests/test_simulation_host.py"]

PLANTS = [
    ("phase of the transform with the wrong sign",
     "phase = np.exp(1j * (np.asarray(k, dtype=np.float64) @ Rv.T))",
     "phase = np.exp(-1j * (np.asarray(k, dtype=np.float64) @ Rv.T))"),
    ("1/N_cell dropped",
     'S = np.einsum("kd,...dab->...kab", phase, Cd) / float(n_cells)',
     'S = np.einsum("kd,...dab->...kab", phase, Cd)'),
    ("orbitals a, b transposed",
     'S = np.einsum("kd,...dab->...kab", phase, Cd) / float(n_cells)',
     'S = np.einsum("kd,...dab->...kba", phase, Cd) / float(n_cells)'),
    ("background subtracted at every momentum",
     "S = S - zero[:, None, None] * back[..., None, :, :]",
     "S = S - back[..., None, :, :]"),
    ("background N_cell <O_a><O_b> without N_cell",
     "back = float(n_cells) * O[..., :, None] * O[..., None, :]",
     "back = O[..., :, None] * O[..., None, :]"),
    ("k quantisation: b_1 from L_1 instead of L_2",
     "b1 = 2.0 * np.pi / d * ((L2 @ g2) * g1 - (L2 @ g1) * g2)",
     "b1 = 2.0 * np.pi / d * ((L1 @ g2) * g1 - (L1 @ g1) * g2)"),
    ("reciprocal vectors without the transpose",
     "G = 2.0 * np.pi * np.linalg.inv(A).T",
     "G = 2.0 * np.pi * np.linalg.inv(A)"),
    ("jackknife error without (N-1)/N",
     "err = np.sqrt((n - 1) / n * ((loo - mean) ** 2).sum(axis=0))",
     "err = np.sqrt(((loo - mean) ** 2).sum(axis=0) / n)"),
    ("jackknife ratio of the left-out bin instead of the rest",
     "loo = (tot_o[None] - os_) / (tot_s - s).reshape(sh)",
     "loo = os_ / s.reshape(sh)"),
    ("rebin keeps the skipped bins",
     "    b = b[n_skip:]\n",
     ""),
]


def _copy_package(dst: str) -> None:
    """The package's Python sources and the tests that exercise the analysis, so
    that the copy (whose conftest puts the copy's root on sys.path) is what runs."""
    for sub, keep in ((PKG, lambda f: f.endswith(".py")),
                      ("tests", lambda f: f in ("__init__.py", "conftest.py") or f in [os.path.basename(t) for t in TESTS])):
        os.makedirs(os.path.join(dst, sub))
        for f in os.listdir(os.path.join(ROOT, sub)):
            if keep(f):
                shutil.copy(os.path.join(ROOT, sub, f), os.path.join(dst, sub, f))


def _run(dst: str) -> int:
    cmd = [sys.executable, "-m", "pytest", *TESTS, "-q", "-x", "-m", "not gpu", "-p", "no:cacheprovider"]
    return subprocess.run(cmd, cwd=dst, capture_output=True, text=True, timeout=600).returncode


def test_unplanted_copy_passes(tmp_path):
    _copy_package(str(tmp_path))
    assert _run(str(tmp_path)) == 0


@pytest.mark.parametrize("name,old,new", PLANTS, ids=[p[0] for p in PLANTS])
def test_planted_mistake_fails_a_test(tmp_path, name, old, new):
    _copy_package(str(tmp_path))
    path = os.path.join(str(tmp_path), PKG, "analysis.py")
    with open(path) as fh:
        src = fh.read()
    assert src.count(old) == 1, old
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    assert _run(str(tmp_path)) == 1, name
