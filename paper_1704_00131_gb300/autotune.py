"""Autotuner of the sweep's launch parameters on this GPU.

For a batch of chains (models and the chain -> model map) it picks, in two
passes:
1. the product kernel family of the reduced-precision path: float-pair SIMT
   register tiles ("mixed") or exact-split BF16 products on the tensor cores
   ("mixed_tc"; the FP64 path has one family, "fp64"), together with the rank k
   of the delayed updates (accepted flips per flush), which sets the shape of the
   flush product (N x k times k x N) and the shared memory the delayed vectors
   take, hence how many CTAs share an SM;
2. for the winner, the tile options: the output tile of the float-pair SIMT
   products (48 x 48 or 64 x 64 per CTA: `dd_tile` 3 or 4) and, with the
   tensor cores, the lattice size from which chains use them (`tc_min_sites`:
   all chains, or the default crossover).

Each candidate runs one untimed sweep of the whole batch, then one sweep timed
with CUDA events on the launching stream; the fastest candidate wins.  All
candidates start from the same seed, so they run the same Markov chains.
Results are cached per (GPU name, workload signature) in a JSON file.

The selection and cache logic (`choose`, `signature`, `Cache`) are plain host
code; `tune` is the only part that launches work, through the C ABI.
"""
from __future__ import annotations

import hashlib
import json
import os
from dataclasses import dataclass, field

import numpy as np

DEFAULT_DELAYS = (8, 16, 24, 32)
FAMILIES = {"mixed": ("mixed", "mixed_tc"), "mixed_tc": ("mixed", "mixed_tc"), "fp64": ("fp64",),
            "fp32": ("fp32",)}
DD_TILES = (3, 4)
TC_MIN_SITES = (1, 0)   # every chain on the tensor cores; the library's default crossover


@dataclass
class Choice:
    precision: str
    delay_k: int
    ms: float
    timings: list = field(default_factory=list)   # [(precision, delay_k, options, ms)]
    cached: bool = False
    options: dict = field(default_factory=dict)   # run options: dd_tile, tc_min_sites

    def as_dict(self) -> dict:
        return {"precision": self.precision, "delay_k": self.delay_k, "ms": self.ms, "options": dict(self.options),
                "timings": [list(t) for t in self.timings], "cached": self.cached}


def option_candidates(precision: str) -> list:
    """Tile options tried for the winner of the first pass."""
    if precision not in ("mixed", "mixed_tc"):
        return []
    out = [{"dd_tile": t} for t in DD_TILES]
    if precision == "mixed_tc":
        out += [{"tc_min_sites": m} for m in TC_MIN_SITES]
    return out


def candidates(precision: str, delays=DEFAULT_DELAYS) -> list:
    """(precision, delay_k) pairs of the family that `precision` belongs to."""
    if precision not in FAMILIES:
        raise ValueError(f"unknown precision {precision!r}")
    out = []
    for p in FAMILIES[precision]:
        for k in delays:
            if not 1 <= int(k) <= 64:
                raise ValueError(f"delay_k {k} outside 1..64")
            out.append((p, int(k)))
    return out


def choose(timings) -> tuple:
    """The fastest (precision, delay_k, options, ms) of entries (p, k, ms) or
    (p, k, options, ms); ties go to the earlier candidate."""
    best = None
    for t in timings:
        p, k, opt, ms = (t[0], t[1], {}, t[2]) if len(t) == 3 else t
        if not np.isfinite(ms) or ms <= 0:
            continue
        if best is None or ms < best[3]:
            best = (p, k, dict(opt), ms)
    if best is None:
        raise RuntimeError("no candidate ran")
    return best


def signature(models, chain_model, family: str, delays) -> str:
    """Key of a workload: each chain's (N, M_V, L, n_wrap, field type) and the
    candidate set; the couplings do not change the cost of a sweep."""
    counts = np.bincount(np.asarray(chain_model, dtype=np.int64), minlength=len(models))
    parts = sorted(f"{m.N}/{m.n_vertices}/{m.L}/{m.n_wrap}/{m.field_type}x{int(c)}"
                   for m, c in zip(models, counts) if c)
    text = f"{family}|{','.join(map(str, delays))}|{';'.join(parts)}"
    return hashlib.sha1(text.encode()).hexdigest()[:16]


class Cache:
    """JSON file {device: {signature: choice}}."""

    def __init__(self, path: str | None = None):
        self.path = path or os.path.join(os.environ.get("XDG_CACHE_HOME", os.path.expanduser("~/.cache")),
                                         "dqmc_gb300", "autotune.json")

    def _load(self) -> dict:
        try:
            with open(self.path) as f:
                return json.load(f)
        except (OSError, ValueError):
            return {}

    def get(self, device: str, key: str):
        d = self._load().get(device, {}).get(key)
        if d is None:
            return None
        return Choice(d["precision"], int(d["delay_k"]), float(d["ms"]), [tuple(t) for t in d["timings"]], True,
                      dict(d.get("options", {})))

    def put(self, device: str, key: str, choice: Choice):
        data = self._load()
        data.setdefault(device, {})[key] = choice.as_dict()
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        tmp = f"{self.path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, self.path)


def time_candidate(models, chain_model, precision: str, delay_k: int, seed: int, stream=None, **options) -> float:
    """Milliseconds of one sweep of the batch (after one untimed sweep)."""
    import torch

    from . import dqmc
    st = stream if stream is not None else torch.cuda.current_stream()
    ens = dqmc.Ensemble(models, chain_model, precision=precision, delay_k=delay_k, seed=seed, stream=st, **options)
    try:
        ens.sweep(1, stats=False)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        ens.sweep(1, stats=False)
        b.record(st)
        torch.cuda.synchronize()
        return float(a.elapsed_time(b))
    finally:
        ens.close()


def tune(models, chain_model, precision: str = "mixed", delays=DEFAULT_DELAYS, seed: int = 0, stream=None,
         cache: Cache | None = None, timer=None, device: str | None = None) -> Choice:
    """Pick (precision variant, delay_k) for this batch on this GPU.

    `timer(models, chain_model, precision, delay_k, seed, stream) -> ms` defaults
    to `time_candidate`; `cache=None` disables the cache."""
    if device is None:
        import torch
        device = torch.cuda.get_device_name(torch.cuda.current_device())
    key = signature(models, chain_model, FAMILIES[precision][0], tuple(delays))
    if cache is not None:
        hit = cache.get(device, key)
        if hit is not None:
            return hit
    run = timer or time_candidate
    timings = []
    for p, k in candidates(precision, delays):
        timings.append((p, k, {}, float(run(models, chain_model, p, k, seed, stream))))
    p, k, opt, ms = choose(timings)
    for o in option_candidates(p):
        timings.append((p, k, o, float(run(models, chain_model, p, k, seed, stream, **o))))
    p, k, opt, ms = choose(timings)
    ch = Choice(p, k, ms, timings, False, opt)
    if cache is not None:
        cache.put(device, key, ch)
    return ch
