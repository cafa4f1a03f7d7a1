#!/usr/bin/env python
"""Throughput of the batched DQMC sweep on GB300: field-update proposals/s and sweeps/s.

One step = one sweep (tau = 1..L and back) of every chain of the workload.
Default workload: 256 independent chains of the square-lattice Hubbard model,
half 8x8 (N = 64) and half 12x12 (N = 144), beta = 4 or 8 (dtau = 0.1), U in
{2, 4, 6}, spin-z Ising decoupling, n_wrap = 10; fields drawn from Philox.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64|fp32]
    python bench.py --impl reference     # the FP64 CPU oracle on the host cores

Multi-GPU (torchrun): every rank runs its own batch of chains (independent
Markov chains, no data-path collective); value = all ranks' proposals / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1704_00131_gb300 import workloads as W  # noqa: E402

METRIC = "field-update proposals/s (and sweeps/s) of the batched DQMC sweep at max|dG|<=1e-6"
UNIT = "proposals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c3", choices=["c1", "c2", "c3", "c5"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "fp32", "mixed", "mixed_tc"])
    ap.add_argument("--chains", type=int, default=0, help="override the number of chains (c3/c5)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true", help="skip timing the plain FP64 path")
    ap.add_argument("--peaks", action="store_true", help="measure the matmul peaks used as roofline denominators")
    ap.add_argument("--no-oracle-check", action="store_true", help="skip the max|dG| check against the oracle")
    ap.add_argument("--gradients", action="store_true",
                    help="time the log-det and energy adjoints of the 64-configuration 8x8, beta = 4 workload")
    ap.add_argument("--paper-example", action="store_true",
                    help="precision monitors of the paper's 4x4, U=4, beta=10 spin-z example instead of the bench")
    ap.add_argument("--run-option", action="append", default=[], metavar="KEY=VALUE",
                    help="a dqmc_run_opts field for the main path without the autotuner (e.g. tc_min_sites=1)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use --precision and the workload's delay_k as given instead of tuning them")
    return ap.parse_args()


def workload(name: str, chains: int = 0) -> W.Workload:
    if chains and name == "c3":
        return W.config_c3(chains)
    if chains and name == "c5":
        return W.config_c5(chains)
    return {"c1": W.config_c1, "c2": W.config_c2, "c3": W.config_c3, "c5": W.config_c5}[name]()


def chain_cost(m: W.ModelSpec, accepted_per_chain: float) -> float:
    """Algorithmic FLOPs of one sweep of one chain (two flavors):
    wraps 2 flavors x 2L slices x 2 GEMMs x 2N^3; accepted flips 2 flavors x 2N^2;
    stabilisation 2 flavors x 2L/n_wrap events x (2 n_wrap + 37/3) N^3
    (B-chain GEMMs, QR 4/3, form Q 4/3, T update 1, Q^T Q 2, T T^T 2, LU 2/3,
    solve 2, Q X 2)."""
    N, L, nw = m.N, m.L, m.n_wrap
    nfl = m.hopping.shape[0]
    wraps = nfl * 2 * L * 2 * 2 * N ** 3
    upd = nfl * accepted_per_chain * 2 * N ** 2
    stab = nfl * (2 * L // nw) * (2 * nw + 37.0 / 3.0) * N ** 3
    return wraps + upd + stab


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
                for i, n in enumerate(names):
                    if r[3 + i].strip().lower() == "active":
                        reasons.add(n)
            except Exception:
                continue
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# ----------------------------------------------------------------- CPU oracle
def oracle_sample(wl: W.Workload, n_threads: int, per_class: int):
    """Time the FP64 oracle (one sweep per chain) on a stratified sample of the
    workload's chains, run concurrently on n_threads host threads (ctypes releases
    the GIL).  Returns (proposals, seconds, description)."""
    import oracle
    oracle.build()
    classes = {}
    for c, mi in enumerate(wl.chain_model):
        classes.setdefault(int(mi), []).append(c)
    sample = []
    for mi, cs in sorted(classes.items()):
        sample += [(mi, c) for c in cs[:per_class]]
    chains = []
    for mi, c in sample:
        m = wl.models[mi]
        om = oracle.Model(m.hopping, m.vertex_site, m.vertex_sign, m.U, m.dtau, m.L, m.n_wrap, m.field_type)
        chains.append((oracle.Chain(om, None, seed=W.BASE_SEED, chain=c), 2 * m.L * m.n_vertices))
    idx = [0]
    lock = threading.Lock()
    errors = []

    def worker():
        while True:
            with lock:
                if idx[0] >= len(chains):
                    return
                i = idx[0]
                idx[0] += 1
            try:
                chains[i][0].sweep(1)
            except BaseException as e:       # a failed chain must not be counted as swept
                with lock:
                    errors.append(e)
                return

    t0 = time.perf_counter()
    n_threads = max(1, min(n_threads, len(chains)))       # threads that get work
    th = [threading.Thread(target=worker) for _ in range(n_threads)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    dt = time.perf_counter() - t0
    if errors:
        raise RuntimeError(f"oracle baseline: {len(errors)} of {len(chains)} chain sweeps failed") from errors[0]
    props = sum(p for _, p in chains)
    desc = (f"1 sweep each of {len(chains)} chains ({per_class} per model class of the workload: "
            + ", ".join(f"{wl.models[mi].name}" for mi in sorted(classes)) + f") on {n_threads} threads")
    return props, dt, desc, n_threads


def run_reference(args, wl: W.Workload, rank: int):
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    n_cls = max(1, len(set(wl.chain_model.tolist())))
    per_class = max(1, -(-cores // n_cls))                   # enough chains to give every core work
    for _ in range(args.warmup):
        oracle_sample(wl, cores, 1)
    times, props = [], 0
    desc, used = "", cores
    for _ in range(args.steps):
        p, dt, desc, used = oracle_sample(wl, cores, per_class)
        times.append(dt)
        props = p
    tot = sum(times)
    value = props * args.steps / tot
    sweeps_per_s = value / wl.proposals_per_sweep()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Philox fields)",
        "config": {"workload": wl.name, "chains": wl.n_chains, "sample": desc},
        "sweeps_per_s": sweeps_per_s,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------- rank helpers
def rank_seed(rank: int) -> int:
    """Each rank runs its own independent chains (the paper's one walker per task)."""
    return W.BASE_SEED + rank


def max_over_ranks(ms: float, device="cuda") -> float:
    """The slowest rank sets the time of a step (the only collective, outside the data path)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(proposals_per_step: int, world: int, ms_step: float) -> float:
    """Proposals of all ranks per second of the slowest rank."""
    return proposals_per_step * world / (ms_step / 1000.0)


# ---------------------------------------------------------------------- ours
# A float-pair (double-word) multiply-add costs 12 FP32-pipe operations
# (TwoProd by FMA, TwoSum, two cross-term FMAs, accumulation).
DW_OPS_PER_FMA = 12.0
# An exact-split product spends 28 BF16 digit-pair products (seven digits per
# operand, diagonals t + u <= 6) on every multiply-add.
SPLIT_PRODUCTS = 28.0

# DRAM bytes (read + write) per launch of the sweep kernel from one ncu capture,
# valid only for the kernel sources it was taken on: keyed by (precision,
# workload, delay_k) -> (sha256 prefix of the kernel sources, bytes).  A source
# change makes the lookup miss and the line report traffic null.  Capture:
# `ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
# --clock-control none -k regex:sweep_kernel -s 3 -c 1` on the full 256-chain
# workload with the tensor-core products (34.54 GB read, 88.39 GB written).
TRAFFIC_BYTES = {("mixed_tc", "square 8x8/12x12 x256 chains", 16): ("bdde3c910e225dba", 122932378368)}

KERNEL_SOURCES = ["dqmc_device.cuh", "dqmc_umma.cuh", "dqmc_internal.h", "dqmc_sweep_fp64.cu",
                  "dqmc_sweep_fp32.cu", "dqmc_sweep_mixed.cu", "dqmc_sweep_mixed_tc.cu"]


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1704_00131_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    """Roofline denominators measured in this process (cuBLAS through torch, best
    of a few launches): FP64 and FP32-SIMT matmul rates; the BF16 tensor rate from
    the driver's MEASURED_PEAKS.json when present."""
    import torch

    def rate(dtype, n, iters):
        a = torch.randn(n, n, device="cuda", dtype=dtype)
        b = torch.randn(n, n, device="cuda", dtype=dtype)
        for _ in range(2):
            a @ b
        torch.cuda.synchronize()
        best = 0.0
        for _ in range(iters):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            a @ b
            s1.record()
            torch.cuda.synchronize()
            best = max(best, 2 * n ** 3 / (s0.elapsed_time(s1) * 1e-3) / 1e12)
        return best

    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {"fp64_tflops": rate(torch.float64, 4096, 3), "fp32_simt_tflops": rate(torch.float32, 8192, 5),
           "source": "cuBLAS DGEMM 4096^3 / SGEMM 8192^3 (TF32 off) measured in this run, best of 3 / 5"}
    torch.backends.cuda.matmul.allow_tf32 = tf32
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        out["bf16_tflops_sustained"] = float(mp["bf16_tflops_sustained"])
        out["bf16_source"] = "MEASURED_PEAKS.json (cuBLAS bf16, sustained)"
    except Exception:
        out["bf16_tflops_sustained"] = 1700.0
        out["bf16_source"] = "fallback (no MEASURED_PEAKS.json)"
    return out


def time_path(wl, precision, args, stream, seed, world, local_rank, delay_k=None, peaks=None, options=None):
    """Warm up, then time args.steps sweeps of every chain with CUDA events."""
    import torch

    from paper_1704_00131_gb300 import dqmc
    ens = dqmc.Ensemble(wl.models, wl.chain_model, precision=precision, delay_k=delay_k or wl.delay_k, seed=seed,
                        stream=stream, **(options or {}))
    ens.sweep(max(args.warmup - 1, 0), stats=False)
    st = ens.sweep(1)
    acc_per_chain = st["accepted"] / wl.n_chains
    flops_per_step = sum(chain_cost(wl.models[m], acc_per_chain) for m in wl.chain_model)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local_rank) as clk:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for i in range(args.steps):
            ev[i][0].record(stream)
            ens.sweep(1, stats=False)
            ev[i][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
    ms_total = t_start.elapsed_time(t_end)
    per_launch_ms = [a.elapsed_time(b) for a, b in ev]
    ms_total = max_over_ranks(ms_total)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ms_step = ms_total / args.steps
    value = whole_job_value(wl.proposals_per_sweep(), world, ms_step)
    avg_launch_s = statistics.mean(per_launch_ms) / 1000.0
    achieved = flops_per_step / avg_launch_s / 1e12
    pk = peaks or {}
    if precision == "fp64":
        bound, peak, kern = "alu", pk.get("fp64_tflops"), "sweep_kernel<double>"
        src = "FP64 pipe: " + pk.get("source", "")
    elif precision == "fp32":
        bound, peak, kern = "alu", pk.get("fp32_simt_tflops"), "sweep_kernel<float>"
        src = "FP32 SIMT pipe: " + pk.get("source", "")
    elif precision == "mixed_tc":
        bound, kern = "tensor", "sweep_kernel<dd> (tcgen05 split-BF16 products)"
        peak = pk.get("bf16_tflops_sustained", 0.0) / SPLIT_PRODUCTS if pk else None
        src = ("BF16 tensor peak / 28 digit-pair products per multiply-add (" + pk.get("bf16_source", "") +
               "); only the N^3 products run on the tensor cores, the QR, LU, solves and updates on the "
               "FP32 pipes in float pairs")
    else:
        bound, kern = "alu", "sweep_kernel<dd>"
        peak = pk.get("fp32_simt_tflops", 0.0) / DW_OPS_PER_FMA if pk else None
        src = ("double-word arithmetic on the FP32 pipes: SGEMM rate / 12 FP32 operations per float-pair "
               "multiply-add (" + pk.get("source", "") + ")")
    hit = TRAFFIC_BYTES.get((precision, wl.name, delay_k or wl.delay_k))
    srchash = kernel_source_hash()
    traffic = hit[1] if hit and hit[0] == srchash else None
    roof = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if peak else None, "traffic": traffic,
            "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
            "traffic_note": ("ncu capture on these kernel sources" if traffic is not None else
                             f"no ncu capture on these kernel sources (sha {srchash})"),
            "kernel": kern, "peak_source": src}
    if precision == "mixed_tc" and pk.get("fp32_simt_tflops"):
        # the same launch against the double-word peak of the FP32 pipes, where
        # everything but the N^3 products runs
        roof["frac_double_word"] = achieved / (pk["fp32_simt_tflops"] / DW_OPS_PER_FMA)
    return {"ens": ens, "st": st, "ms_step": ms_step, "value": value, "roofline": roof, "clocks": clk.summary(),
            "algorithmic_tflop_per_step": flops_per_step / 1e12}


def oracle_checks(wl, ens, n_threads):
    """Accuracy of a path against the FP64 oracle on the GPU's current fields, one
    chain per model class of the workload (flavor up):
    * fresh_G0: max |G_GPU(0) - G_oracle(0)| of the working G after the sweeps
      (a stable recompute at the end of every sweep);
    * wrapped_interior: max |G_wrap(tau) - G_oracle(tau)| at tau = L/2 - 1, n_wrap - 1
      slices after a stabilisation point, with G_wrap the path's own wrapped G on
      frozen fields (dqmc_greens_tau);
    * oracle_nwrap_sensitivity: max |G_oracle(tau; n_wrap) - G_oracle(tau; n_wrap / 2)|
      at the same tau, the FP64 oracle's own round-off amplification at that
      conditioning."""
    import oracle
    oracle.build()
    fields, _ = ens.get_fields()
    picks = {}
    for c, mi in enumerate(wl.chain_model):
        picks.setdefault(int(mi), c)
    jobs = []
    for mi, c in sorted(picks.items()):
        m = wl.models[mi]
        om = oracle.Model(m.hopping, m.vertex_site, m.vertex_sign, m.U, m.dtau, m.L, m.n_wrap, m.field_type)
        om2 = oracle.Model(m.hopping, m.vertex_site, m.vertex_sign, m.U, m.dtau, m.L, max(1, m.n_wrap // 2),
                           m.field_type)
        jobs.append((om, om2, fields[c], c, m.L // 2 - 1))
    res = [None] * len(jobs)
    errors = []

    def work(i):
        om, om2, f, c, ti = jobs[i]
        try:
            res[i] = (oracle.green_udv(om, f, 0, 0)[0], oracle.green_udv(om, f, 0, ti)[0],
                      oracle.green_udv(om2, f, 0, ti)[0])
        except BaseException as e:
            errors.append(e)

    ths = []
    for i in range(len(jobs)):
        t = threading.Thread(target=work, args=(i,))
        t.start()
        ths.append(t)
        if len(ths) >= n_threads:
            for t in ths:
                t.join()
            ths = []
    for t in ths:
        t.join()
    if errors:
        raise RuntimeError(f"oracle accuracy check: {len(errors)} of {len(jobs)} oracle recomputes failed") from errors[0]
    fresh = wrapped = delta = 0.0
    for i, (_, _, _, c, ti) in enumerate(jobs):
        G0, Gt, Gt2 = res[i]
        fresh = max(fresh, float(np.abs(ens.greens(c, 0)[0] - G0).max()))
        wrapped = max(wrapped, float(np.abs(ens.greens_tau(c, 0, ti) - Gt).max()))
        delta = max(delta, float(np.abs(Gt - Gt2).max()))
    return {"fresh_G0_max_abs_dG": fresh, "wrapped_interior_max_abs_dG": wrapped,
            "oracle_nwrap_sensitivity": delta, "chains_checked": len(jobs)}


def run_ours(args, wl: W.Workload, rank: int, world: int, local_rank: int):
    import torch

    from paper_1704_00131_gb300 import build_ext

    build_ext.build()
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    seed = rank_seed(rank)
    peaks = measured_peaks()
    main_prec, k_main, k_fp64 = args.precision, wl.delay_k, wl.delay_k
    opt_main = {k: int(v) for k, v in (o.split("=", 1) for o in args.run_option)}
    tuned = None
    if not args.no_autotune:
        # untimed: pick the product family and the delayed-update rank on this GPU
        from paper_1704_00131_gb300 import autotune
        ch = autotune.tune(wl.models, wl.chain_model, args.precision, seed=seed, stream=stream, cache=None)
        main_prec, k_main, opt_main = ch.precision, ch.delay_k, dict(ch.options)
        tuned = {"main": ch.as_dict()}
        if main_prec != "fp64" and not args.no_fp64_compare:
            cf = autotune.tune(wl.models, wl.chain_model, "fp64", seed=seed, stream=stream, cache=None)
            k_fp64 = cf.delay_k
            tuned["fp64"] = cf.as_dict()
    r = time_path(wl, main_prec, args, stream, seed, world, local_rank, delay_k=k_main, peaks=peaks,
                  options=opt_main)
    ens, st = r["ens"], r["st"]
    props_step = wl.proposals_per_sweep()
    # end to end through the public API with host buffers: fields in (pinned host),
    # one sweep, fields and measurements out, every step
    fields, ctr = ens.get_fields()
    flat = np.concatenate([f.ravel() for f in fields])
    pinned = torch.from_numpy(flat).pin_memory()
    h2d = int(pinned.numel())
    offs = np.cumsum([0] + [f.size for f in fields])
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        host_fields = np.asarray(pinned.numpy())
        ens.set_fields([host_fields[offs[c]:offs[c + 1]] for c in range(len(fields))], ctr)
        ens.sweep(1, stats=False)
        fields, ctr = ens.get_fields()
        meas = ens.measure()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(1000.0 * (time.perf_counter() - t0) / e2e_steps) / 1000.0   # slowest rank
    d2h = int(sum(f.size for f in fields) + sum(a.nbytes for a in meas))
    e2e_value = props_step * world / e2e_s
    dg = None
    cores = os.cpu_count() or 1
    if rank == 0 and not args.no_oracle_check:
        dg = oracle_checks(wl, ens, cores)
    ens.close()
    fp64 = None
    if main_prec != "fp64" and not args.no_fp64_compare:
        rf = time_path(wl, "fp64", args, stream, seed, world, local_rank, delay_k=k_fp64, peaks=peaks)
        dg64 = oracle_checks(wl, rf["ens"], cores) if (rank == 0 and not args.no_oracle_check) else None
        rf["ens"].close()
        fp64 = {"value": rf["value"], "unit": UNIT, "ms_per_step": rf["ms_step"], "delay_k": k_fp64,
                "accuracy": dg64,
                "roofline": rf["roofline"],
                "critical_chain_ms": {k: round(rf["st"][k], 3) for k in ("ms_update", "ms_wrap", "ms_stab")},
                "prec_green_max": rf["st"]["prec_green_max"], "prec_green_mean": rf["st"]["prec_green_mean"]}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_cls = max(1, len(set(wl.chain_model.tolist())))
        p, dt, desc, used = oracle_sample(wl, cores, max(1, -(-cores // n_cls)))
        cpu = {"value": p / dt, "unit": UNIT, "cores": used, "kind": "oracle", "sample": desc}
    if rank == 0:
        line = {
            "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32+f64", "mixed": "f32x2+f64", "mixed_tc": "bf16-split+f32x2+f64"}[main_prec],
            "data": "synthetic (seeded Philox fields, random-init Markov chains)",
            "config": {"workload": wl.name, "chains": wl.n_chains, "precision": main_prec,
                       "delay_k": k_main, "run_options": opt_main, "n_wrap": 10, "autotune": tuned,
                       "l2": "resident state > L2 (per-chain G, UDV storage and workspace, "
                             f"{ens_bytes(wl, main_prec) / 1e9:.2f} GB); no flush"},
            "sweeps_per_s": 1000.0 / r["ms_step"] * world,
            "accept_rate": st["accepted"] / st["proposals"],
            "accuracy": dg,
            "peaks": peaks,
            "prec_green_max": st["prec_green_max"], "prec_green_mean": st["prec_green_mean"],
            "critical_chain_ms": {k: round(st[k], 3) for k in ("ms_update", "ms_wrap", "ms_stab", "ms_measure")},
            "critical_chain_detail_ms": dict(zip(("ratio_precompute", "accept_scan", "update_vectors", "flushes",
                                                  "b_chain", "qr_and_q", "t_update", "stable_green"),
                                                 [round(x, 3) for x in st["ms_detail"]])),
            "algorithmic_tflop_per_step": r["algorithmic_tflop_per_step"],
            "gpu_launches": 2 * args.steps,
            "roofline": r["roofline"],
            "fp64_path": fp64,
            "speedup_vs_fp64_path": (r["value"] / fp64["value"]) if fp64 else None,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "clocks": r["clocks"],
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def ens_bytes(wl: W.Workload, precision: str) -> float:
    rs = 4 if precision == "fp32" else 8
    tot = 0
    for m in wl.chain_model:
        mm = wl.models[m]
        N, L, nw = mm.N, mm.L, mm.n_wrap
        ld = (N + 3) // 4 * 4
        per_fl = 2 * N * ld * rs + (L // nw + 1) * (2 * N * ld + ld) * 8 + (10 * N * ld + 8 * ld) * 8
        tot += 2 * per_fl + L * mm.n_vertices
    return float(tot)


def measure_peaks():
    """cuBLAS matmul rates (torch) of this GPU: the roofline denominators."""
    import torch
    res = {}

    def rate(dtype, n, tf32=False, iters=10):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, device="cuda", dtype=dtype)
        b = torch.randn(n, n, device="cuda", dtype=dtype)
        for _ in range(3):
            a @ b
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record()
        for _ in range(iters):
            a @ b
        s1.record()
        torch.cuda.synchronize()
        return 2 * n ** 3 / (s0.elapsed_time(s1) / iters * 1e-3) / 1e12

    res["fp64_tflops"] = rate(torch.float64, 8192, iters=5)
    res["fp32_simt_tflops"] = rate(torch.float32, 8192)
    res["tf32_tflops"] = rate(torch.float32, 8192, tf32=True)
    res["bf16_tflops"] = rate(torch.bfloat16, 8192)
    res["device"] = torch.cuda.get_device_name(0)
    print(json.dumps(res), flush=True)


def paper_example(args):
    """The numerical-precision example the paper prints for the spin-z decoupling
    (Sec. 6, 4x4 square lattice, U/t = 4, beta t = 10; here dtau = 0.1, n_wrap = 10):
    the "Precision Green" and "Precision tau" monitors (mean, max) of the FP64 and
    mixed paths over args.steps sweeps after args.warmup, with the time-displaced
    functions measured after every sweep, next to the values of the paper's info file;
    then the same for the SU(2) decoupling's example (Sec. 6.1), with its
    "Precision Phase", the Precision tau of one time-displaced measurement over
    the whole interval after the sweeps, and the throughput of a batch of its
    chains."""
    from paper_1704_00131_gb300 import build_ext, dqmc
    build_ext.build()
    m = W.ModelSpec(W.square_lattice(4, 4), U=4.0, dtau=0.1, L=100, n_wrap=10, name="square4x4_U4_b10")
    out = {"workload": m.name, "sweeps": args.steps, "warmup": args.warmup,
           "paper_info_file": {"precision_green_mean_max": [5.0823874429126405e-11, 5.8621144596315844e-06],
                               "precision_tau_mean_max": [1.5929357848647394e-11, 1.0985132530727526e-05]}}
    for prec in ("fp64", "mixed"):
        ens = dqmc.Ensemble([m], [0], precision=prec, delay_k=16, seed=W.BASE_SEED)
        ens.sweep(args.warmup, stats=False)
        gm, gx, tm, tx = [], 0.0, [], 0.0
        for _ in range(args.steps):
            st = ens.sweep(1)
            gm.append(st["prec_green_mean"])
            gx = max(gx, st["prec_green_max"])
            _, _, pt = ens.measure_tau(m.L)
            tm.append(pt[0])
            tx = max(tx, pt[1])
        ens.close()
        out[prec] = {"precision_green_mean_max": [float(np.mean(gm)), gx],
                     "precision_tau_mean_max": [float(np.mean(tm)), tx]}
    # the SU(2) charge decoupling example of Sec. 6.1 (same lattice and couplings):
    # Precision Green and Precision Phase, and the throughput of a batch of chains
    n_su2 = args.chains if args.chains > 0 else 304
    ms2 = dqmc.Su2Model(W.square_lattice(4, 4), U=4.0, dtau=0.1, L=100, n_wrap=10)
    ens = dqmc.Su2Ensemble([ms2], [0] * n_su2, seed=W.BASE_SEED)
    ens.sweep(args.warmup)
    st = ens.sweep(args.steps)
    _, pt = ens.measure_tau(ms2.L)
    ens.close()
    out["su2"] = {"workload": f"su2_square4x4_U4_b10 x {n_su2} chains",
                  "paper_info_file": {"precision_green_mean_max": [1.2918865817224671e-14, 4.0983018995027644e-11],
                                      "precision_phase_max": 5.0272908791449966e-12,
                                      "precision_tau_mean_max": [8.4596701790588625e-15, 3.5033530012121281e-11]},
                  "precision_green_mean_max": [st["prec_green_mean"], st["prec_green_max"]],
                  "precision_phase_max": st["prec_phase_max"],
                  "precision_tau_mean_max": [pt[0], pt[1]], "mean_sign": st["mean_sign"],
                  "acceptance": st["accepted"] / st["proposals"],
                  "proposals_per_s": st["proposals"] / (st["ms_total"] * 1e-3),
                  "ms_per_sweep": st["ms_total"] / args.steps, "dtype": "complex f64"}
    print(json.dumps(out), flush=True)


def gradients(args):
    """The differentiation workload: d log|det(1+B(beta,0))| / d(K, U) and
    d Ener / d(K, U) on square 8x8 (N = 64), beta = 4 (L = 40), U = 4, for 64
    seeded field configurations, FP64 (the adjoint of Sec. 2.3's B chain,
    checkpointed at the stabilisation points).  Prints one JSON line: configurations
    per second for both adjoints together (device time, CUDA events, after
    warm-up), the gradients of one configuration against the FP64 oracle, and the
    oracle's own time for that configuration on one host core."""
    import torch

    import oracle
    from paper_1704_00131_gb300 import build_ext, dqmc
    build_ext.build()
    torch.cuda.set_device(0)
    m = W.ModelSpec(W.square_lattice(8, 8), U=4.0, dtau=0.1, L=40, n_wrap=10, name="square8x8_U4_b4")
    f = np.stack([W.random_fields(1, m.L, m.n_vertices, seed=s) for s in range(1, 65)])
    ens = dqmc.Ensemble([m], [0], precision="fp64")
    for _ in range(max(1, args.warmup)):
        ens.logdet_backward(0, f[:8])
        ens.energy_backward(0, f[:8])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.steps):
        ld, gKl, gUl = ens.logdet_backward(0, f)
        e, gKe, gUe = ens.energy_backward(0, f)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    om = oracle.Model(m.hopping, m.vertex_site, m.vertex_sign, m.U, m.dtau, m.L, m.n_wrap, m.field_type)
    t0 = time.perf_counter()
    ldo, _, gKlo, gUlo = oracle.logdet_grad(om, f[0])
    eo, gKeo, gUeo = oracle.energy_grad(om, f[0])
    t_orc = time.perf_counter() - t0
    ens.close()
    dev = {"logdet": float(np.max(np.abs(ld[0] - ldo) / np.maximum(1.0, np.abs(ldo)))),
           "dlogdet_dK": float(np.max(np.abs(gKl[0] - gKlo))), "dlogdet_dU": float(np.max(np.abs(gUl[0] - gUlo))),
           "ener": float(np.max(np.abs(e[0] - eo))), "dener_dK": float(np.max(np.abs(gKe[0] - gKeo))),
           "dener_dU": float(abs(gUe[0] - gUeo))}
    print(json.dumps({"metric": "gradient configurations/s (log-det and energy adjoints together)",
                      "value": 64.0 / (ms * 1e-3), "unit": "configurations/s", "ms_per_step": ms,
                      "steps": args.steps, "warmup": args.warmup, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": m.name + " x 64 configurations", "n_wrap": m.n_wrap},
                      "max_abs_dev_vs_oracle_config0": dev,
                      "cpu_baseline": {"value": 1.0 / t_orc, "unit": "configurations/s", "cores": 1,
                                       "kind": "oracle", "sample": "both adjoints of configuration 0"}}),
          flush=True)


def main():
    args = parse()
    if args.gradients:
        gradients(args)
        return
    if args.peaks:
        measure_peaks()
        return
    if args.paper_example:
        paper_example(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    wl = workload(args.config, args.chains)
    if args.impl == "reference":
        run_reference(args, wl, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_ours(args, wl, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
