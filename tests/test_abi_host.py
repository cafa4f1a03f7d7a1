"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a,
loads, exports every entry point that include/dqmc.h declares, and refuses to
run without a CUDA device instead of falling back to the CPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1704_00131_gb300 import build_ext, dqmc
from paper_1704_00131_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return dqmc.load()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(dqmc_[a-z_0-9]+)\s*\(", txt))
    return names


def test_header_declares_the_named_entry_points():
    names = declared_symbols()
    for n in ("dqmc_init", "dqmc_sweep", "dqmc_greens", "dqmc_measure", "dqmc_logdet_backward"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_symbols():
        assert hasattr(lib, n), n


def test_no_cpu_fallback_without_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = W.ModelSpec(W.square_lattice(2, 2), U=2.0, dtau=0.1, L=4, n_wrap=2)
    with pytest.raises(dqmc.DqmcError) as e:
        dqmc.Ensemble([m], [0])
    assert e.value.status == dqmc.DQMC_ECUDA


def test_invalid_model_rejected_before_any_device_work(lib):
    m = W.ModelSpec(W.square_lattice(2, 2), U=2.0, dtau=0.1, L=5, n_wrap=2)  # L % n_wrap != 0
    with pytest.raises(dqmc.DqmcError) as e:
        dqmc.Ensemble([m], [0])
    assert e.value.status == dqmc.DQMC_EINVAL
    K = W.square_lattice(2, 2)
    K[0, 1] += 0.5  # not symmetric
    with pytest.raises(dqmc.DqmcError) as e:
        dqmc.Ensemble([W.ModelSpec(K, U=2.0, dtau=0.1, L=4, n_wrap=2)], [0])
    assert e.value.status == dqmc.DQMC_EINVAL


def test_invalid_options_rejected_before_any_device_work(lib):
    m = W.ModelSpec(W.square_lattice(2, 2), U=2.0, dtau=0.1, L=4, n_wrap=2)
    for kw in ({"spin_limit": -1}, {"delay_k": 0}, {"delay_k": 65}):
        with pytest.raises(dqmc.DqmcError) as e:
            dqmc.Ensemble([m], [0], **kw)
        assert e.value.status == dqmc.DQMC_EINVAL, kw


def test_su2_context_has_no_cpu_fallback_and_validates_on_the_host(lib):
    """The complex family: without a device the context fails with DQMC_ECUDA (no
    CPU path); invalid models, bonds and J pairs are rejected with DQMC_EINVAL
    before any device work."""
    import torch
    K = W.chain_lattice(3)
    good = dqmc.Su2Model(K, U=2.0, dtau=0.1, L=4, n_wrap=2, bonds=[(0, 1), (1, 2)], xi=0.5, h=1.0, pairs=[(0, 1)])
    if not torch.cuda.is_available():
        with pytest.raises(dqmc.DqmcError) as e:
            dqmc.Su2Ensemble([good], [0])
        assert e.value.status == dqmc.DQMC_ECUDA
    bad = [dict(L=5), dict(bonds=[(0, 0)], h=1.0), dict(bonds=[(0, 3)], h=1.0), dict(bonds=[(0, 1)], h=0.0),
           dict(bonds=[(0, 1)], h=1.0, pairs=[(0, 0)]), dict(pairs=[(0, 1)])]
    for kw in bad:
        args = dict(U=2.0, dtau=0.1, L=4, n_wrap=2, xi=0.5)
        args.update(kw)
        with pytest.raises(dqmc.DqmcError) as e:
            dqmc.Su2Ensemble([dqmc.Su2Model(K, **args)], [0])
        assert e.value.status == dqmc.DQMC_EINVAL, kw


def test_svd_stabilisation_needs_the_fp64_path(lib):
    m = W.ModelSpec(W.square_lattice(2, 2), U=2.0, dtau=0.1, L=4, n_wrap=2)
    for prec in ("fp32", "mixed", "mixed_tc"):
        with pytest.raises(dqmc.DqmcError) as e:
            dqmc.Ensemble([m], [0], precision=prec, stab_svd=True)
        assert e.value.status == dqmc.DQMC_EINVAL, prec


def test_binding_lists_every_exported_entry_point(lib):
    assert set(dqmc.EXPORTED) == declared_symbols()


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(dqmc, "_lib", None)
    monkeypatch.setattr(dqmc, "_LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(ImportError):
        dqmc.load()


def test_product_and_oracle_share_no_code():
    """The CUDA path never imports, links or includes the oracle, and the oracle
    imports and includes nothing of the package."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_1704_00131_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn), encoding="utf-8").read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), fn
                assert "dqmc_oracle" not in text and "liboracle" not in text, fn
    for fn in os.listdir(os.path.join(root, "oracle")):
        if fn.endswith((".py", ".c", ".h")):
            text = open(os.path.join(root, "oracle", fn), encoding="utf-8").read()
            assert not re.search(r"^\s*(import|from)\s+paper_1704_00131_gb300\b", text, re.M), fn
            assert not re.search(r"^\s*#\s*include\s*[<\"].*(dqmc|paper_1704)", text, re.M), fn


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes mirrors of the C structs have the header's size and field
    offsets (the header compiled by gcc prints them), so a field added, removed or
    reordered on one side only fails here on the CPU rather than as garbage
    arguments on a GPU."""
    import ctypes
    import json
    import subprocess
    from paper_1704_00131_gb300 import dqmc as dq
    mirrors = {"dqmc_model_desc": dq.ModelDesc, "dqmc_run_opts": dq.RunOpts, "dqmc_sweep_stats": dq.SweepStats,
               "dqmc_su2_model_desc": dq.Su2ModelDesc, "dqmc_su2_opts": dq.Su2Opts,
               "dqmc_su2_sweep_stats": dq.Su2SweepStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dqmc.h"', '#include "dqmc_su2.h"',
             'int main(void) {', '  printf("{");']
    first = True
    for cname, py in mirrors.items():
        fields = ", ".join(f'\\"{f}\\": %zu' for f, _ in py._fields_)
        args = ", ".join(f"offsetof({cname}, {f})" for f, _ in py._fields_)
        sep = "" if first else ", "
        first = False
        lines.append(f'  printf("{sep}\\"{cname}\\": {{\\"sizeof\\": %zu, {fields}}}", sizeof({cname}), {args});')
    lines += ['  printf("}\\n");', '  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    c = json.loads(subprocess.check_output([str(exe)]).decode())
    for cname, py in mirrors.items():
        assert c[cname]["sizeof"] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert c[cname][f] == getattr(py, f).offset, (cname, f)
