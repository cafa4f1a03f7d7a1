"""The reference arm of bench.py on the host cores (no GPU).

`bench.py --impl reference` times the FP64 oracle on the machine's host cores
and prints one JSON line with the same metric, unit and config as the GPU arm;
under torchrun only rank 0 runs it and the other ranks exit without work.  These
tests run it on the 4x4, L = 20 single-chain workload, which the oracle sweeps in
milliseconds.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _json_lines(out: str):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_reference_arm_prints_one_contract_line():
    import bench
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--config", "c1", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 1
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["vs_baseline"] is None
    assert line["dtype"] == "f64"
    wl = bench.workload("c1")
    assert line["config"]["workload"] == wl.name and line["config"]["chains"] == wl.n_chains
    assert line["value"] > 0
    # one sweep of the single chain per step: value = 2 L M_V / (ms_per_step / 1000)
    m = wl.models[0]
    assert line["value"] == pytest.approx(2 * m.L * m.n_vertices / (line["ms_per_step"] / 1000.0), rel=1e-9)
    assert line["sweeps_per_s"] == pytest.approx(line["value"] / wl.proposals_per_sweep(), rel=1e-12)
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["unit"] == line["unit"]
    assert cb["cores"] == 1                      # one chain: one thread gets work
    assert line["config"]["sample"] == cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_under_torchrun_prints_on_rank0_only():
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--config", "c1", "--steps", "1", "--warmup", "0", "--gpus", "2"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    assert lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2 and lines[0]["value"] > 0


def test_oracle_baseline_fails_loudly_when_a_worker_dies(monkeypatch):
    """A host thread of the oracle baseline whose chain raises (the failure is
    injected on the host) stops the run with an error instead of counting that
    chain's proposals as done."""
    import threading
    import bench
    import oracle
    oracle.build()
    real = oracle.Chain.sweep
    calls = {"n": 0}
    lock = threading.Lock()

    def flaky(self, n=1):
        with lock:
            calls["n"] += 1
            k = calls["n"]
        if k == 2:
            raise RuntimeError("injected worker failure")
        return real(self, n)

    import numpy as np
    from paper_1704_00131_gb300 import workloads as W
    monkeypatch.setattr(oracle.Chain, "sweep", flaky)
    m = W.ModelSpec(W.square_lattice(4, 4), U=4.0, dtau=0.1, L=20, n_wrap=10, name="square4x4")
    wl = W.Workload("square 4x4 x4 chains", [m], np.zeros(4, dtype=np.int32), "fp64", 8)
    with pytest.raises(RuntimeError, match="chain sweeps failed"):
        bench.oracle_sample(wl, 2, 4)
    monkeypatch.setattr(oracle.Chain, "sweep", real)
    props, dt, desc, used = bench.oracle_sample(bench.workload("c1"), 2, 1)
    assert props == bench.workload("c1").proposals_per_sweep() and dt > 0 and used == 1
