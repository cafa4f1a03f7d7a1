"""Bins of sweeps and their analysis, the way the paper's main program runs a
simulation (Sec. 5: NBin bins of NSweep sweeps, equal-time and time-displaced
observables accumulated per bin, bin results analysed with the jackknife).

The Markov chains of an `Ensemble` are independent walkers (the paper's one
walker per MPI task); a bin pools the sign-weighted measurements of all chains
over its sweeps.  Everything here is host bookkeeping over the library's
measurement calls: `Ensemble.sweep`, `Ensemble.measure` (energy estimator over
the measurement window), `Ensemble.measure_tau` and `Ensemble.measure_corr`
(one sample per chain after each sweep).

Chained jobs (the paper's configuration files and CPU_MAX): `run` can write a
checkpoint after every bin -- the fields and random-number counter of every
chain and the bins done so far -- and stop once a wall-clock budget is spent; a
later `run` with the same checkpoint on a fresh ensemble of the same models
resumes from it and ends with the same bins as an uninterrupted run.
"""
from __future__ import annotations

import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import analysis


def _sum_over_ranks(raw: dict) -> dict:
    """Sum each array of `raw` over the ranks of the default process group (one
    all-reduce of the concatenated float64 values; CUDA tensors under NCCL)."""
    import torch
    import torch.distributed as dist
    keys = sorted(raw)
    shapes = [np.shape(raw[k]) for k in keys]
    flat = np.concatenate([np.asarray(raw[k], dtype=np.float64).ravel() for k in keys])
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.from_numpy(flat).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    flat = t.cpu().numpy()
    out, off = {}, 0
    for k, sh in zip(keys, shapes):
        n = int(np.prod(sh)) if sh else 1
        out[k] = flat[off:off + n].reshape(sh) if sh else np.float64(flat[off])
        off += n
    return out


@dataclass
class Result:
    """Jackknife mean and error over bins of each sign-reweighted observable."""

    n_bins: int
    sweeps_per_bin: int
    mean_sign: float
    mean: dict = field(default_factory=dict)
    error: dict = field(default_factory=dict)
    cov: dict = field(default_factory=dict)   # N_Cov: covariance of Re S(k, tau) between imaginary times
    complete: bool = True          # False when a time budget stopped the run early


class Simulation:
    """Run `n_bins` bins of `sweeps_per_bin` sweeps after `warmup` sweeps.

    tau:  (n_tau, site_phase per model) -> "gloc_tau" (sum_s,x G(tau,0)_xx per
          site and flavor) and "szz_tau" (sum_xy ph_x ph_y <S^z_x(tau) S^z_y(0)>)
    corr: (pair_class per model, n_class per model) -> "corr_zz", "corr_nn",
          "corr_pm", "corr_gf" per class
    tau_corr: (n_tau, pair_class per model, n_class per model) -> "gf_tau_r",
          "szz_tau_r", "nn_tau_r": sum_s <c_xs(tau) c+_ys(0)>, <S^z_x(tau) S^z_y(0)>
          and <n_x(tau) n_y(0)> per tau and class (`Ensemble.measure_tau_corr`)
    lattice: with `corr` or `tau_corr`, (a1, a2, L1, L2, n_orb, r_cells) of the Bravais
          lattice (unit vectors, periodicity vectors, orbitals per cell and the
          cell displacement of each class, as `workloads.translation_classes_*`
          returns it) -> "corr_zz_k", "corr_nn_k", "corr_pm_k", "corr_gf_k": the
          orbital-resolved S_ab(k) [n_k, n_orb, n_orb] of each correlation at the
          momenta "k" (`analysis.momenta`), Eq. s of Sec. 5.1; the density's
          background N_cell <n_a><n_b> at k = 0 is subtracted with <n_a> from the
          local sum_s <c+ c> of the same bins.  Their error is
          err(Re) + 1j err(Im) (jackknife over bins).  With `tau_corr` likewise
          "gf_tau_k", "szz_tau_k", "nn_tau_k" [n_tau + 1, n_k, n_orb, n_orb], the
          density's background from sum_s G(0,0)_xx = 2 - <n_x>; with n_cov also
          their covariance between imaginary times in `Result.cov`
          [n_tau + 1, n_tau + 1, n_k, n_orb, n_orb] (the paper's N_Cov).
    n_skip, n_rebin: the analysis drops the first n_skip bins and merges every
          n_rebin consecutive bins (the paper's n_skip and N_rebin, Sec. 5.3).
    distributed: one process per GPU, each with its own ensemble (independent
          walkers, the paper's one walker per MPI task): at the end of every bin
          the bin's sums over sweeps and chains are added over all ranks of the
          default torch.distributed group (one all-reduce per bin, the only
          exchange), so every rank analyses the same bins of all chains.  Each
          rank checkpoints its own fields (give each its own path).
    The energy estimator ("kin", "pot", "part", "ener") comes from the ensemble's
    own measurement window (the ensemble must be created with measure=True).
    Chains of different models are pooled, so `tau` and `corr` need a single
    model (or models with the same sizes).
    """

    def __init__(self, ensemble, n_bins: int, sweeps_per_bin: int, warmup: int = 0, tau=None, corr=None,
                 energy: bool = True, lattice=None, tau_corr=None, n_skip: int = 0, n_rebin: int = 1,
                 distributed: bool = False, n_cov: bool = False):
        if n_bins < 2 or sweeps_per_bin < 1 or warmup < 0:
            raise ValueError("need n_bins >= 2, sweeps_per_bin >= 1, warmup >= 0")
        if n_skip < 0 or n_rebin < 1 or (n_bins - n_skip) // n_rebin < 2:
            raise ValueError("need n_skip >= 0, n_rebin >= 1 and two bins left after them")
        if lattice is not None and corr is None and tau_corr is None:
            raise ValueError("lattice needs corr or tau_corr")
        self.ens = ensemble
        self.n_bins = n_bins
        self.sweeps_per_bin = sweeps_per_bin
        self.warmup = warmup
        self.tau = tau
        self.corr = corr
        self.energy = energy
        self.lattice = lattice
        self.tau_corr = tau_corr
        self.n_skip = n_skip
        self.n_rebin = n_rebin
        self.distributed = distributed
        self.n_cov = n_cov
        if distributed:
            import torch.distributed as dist
            if not (dist.is_available() and dist.is_initialized()):
                raise ValueError("distributed needs an initialised torch.distributed process group")

    def _one_bin(self):
        ens = self.ens
        acc, s_acc = {}, 0.0
        if self.energy:
            e0, ss0, n0 = ens.measure()
        for _ in range(self.sweeps_per_bin):
            ens.sweep(1, stats=False)
            sign = None
            if self.tau is not None:
                n_tau, phases = self.tau
                obs, sg, _ = ens.measure_tau(n_tau, phases)
                sign = np.prod(sg, axis=1).astype(np.float64)
                n_sites = np.array([ens.model_of(c).N for c in range(ens.n_chains)], dtype=np.float64)
                nfl = obs.shape[2]
                gloc = obs[:, :, :, 0].sum(axis=2) / (nfl * n_sites[:, None])
                m = obs[..., 0, 2] - obs[..., 1, 2]
                szz = (m * m[..., :1] + obs[..., 0, 1] + obs[..., 1, 1]) / 4.0
                acc["gloc_tau"] = acc.get("gloc_tau", 0.0) + (sign[:, None] * gloc).sum(axis=0)
                acc["szz_tau"] = acc.get("szz_tau", 0.0) + (sign[:, None] * szz).sum(axis=0)
            if self.corr is not None:
                classes, n_class = self.corr
                c, sgc = ens.measure_corr(classes, n_class)
                sgc = sgc.astype(np.float64)
                if sign is None:
                    sign = sgc
                for q, name in enumerate(("corr_zz", "corr_nn", "corr_pm", "corr_gf")):
                    acc[name] = acc.get(name, 0.0) + (sgc[:, None] * c[:, :, q]).sum(axis=0)
            if self.tau_corr is not None:
                n_tau, classes, n_class = self.tau_corr
                o, sgt = ens.measure_tau_corr(n_tau, classes, n_class)
                sgt = sgt.astype(np.float64)
                if sign is None:
                    sign = sgt
                for q, name in enumerate(("gf_tau_r", "szz_tau_r", "nn_tau_r")):
                    acc[name] = acc.get(name, 0.0) + (sgt[:, None, None] * o[..., q]).sum(axis=0)
            if sign is not None:
                s_acc += sign.sum()
        raw = dict(acc)                        # sums over the bin's sweeps and this process's chains
        raw["_s"] = np.float64(s_acc)
        if self.energy:
            e1, ss1, n1 = ens.measure()
            raw["_e"] = (e1 - e0).sum(axis=0)
            raw["_es"] = np.float64((ss1 - ss0).sum())
            raw["_nm"] = np.float64((n1 - n0).sum())
        if self.distributed:
            raw = _sum_over_ranks(raw)         # the chains of every rank in one bin
        out = {k: v / self.sweeps_per_bin for k, v in raw.items() if not k.startswith("_")}
        s_bin = float(raw["_s"]) / self.sweeps_per_bin
        if self.energy and raw["_nm"] > 0:
            de = raw["_e"] / raw["_nm"]                          # sum over chains of sign * O per measurement
            for q, name in enumerate(("kin", "pot", "part", "ener")):
                out[name] = de[q]
            out["_sign_energy"] = float(raw["_es"] / raw["_nm"])
        return out, s_bin

    def _chains_total(self) -> int:
        if not self.distributed:
            return self.ens.n_chains
        return int(round(float(_sum_over_ranks({"n": np.float64(self.ens.n_chains)})["n"])))

    def _save(self, path: str, bins) -> None:
        fields, ctr = self.ens.get_fields()
        data = {"meta": np.array([self.n_bins, self.sweeps_per_bin, self.ens.n_chains, ctr], dtype=np.uint64),
                "signs": np.array([s for _, s in bins], dtype=np.float64)}
        for k in sorted({k for b, _ in bins for k in b}):
            data["bin__" + k] = np.array([b[k] for b, _ in bins])
        for c, f in enumerate(fields):
            data[f"fields__{c}"] = np.asarray(f, dtype=np.int8)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "wb") as fh:
            np.savez(fh, **data)
        os.replace(tmp, path)                  # a crash leaves the previous checkpoint intact

    def _load(self, path: str):
        with np.load(path) as z:
            n_bins, spb, n_chains, ctr = (int(v) for v in z["meta"])
            if (n_bins, spb, n_chains) != (self.n_bins, self.sweeps_per_bin, self.ens.n_chains):
                raise ValueError(f"checkpoint {path} is for {n_bins} bins of {spb} sweeps over {n_chains} chains")
            signs = z["signs"]
            keys = [k[5:] for k in z.files if k.startswith("bin__")]
            cols = {k: z["bin__" + k] for k in keys}
            bins = [({k: cols[k][i] for k in keys}, float(signs[i])) for i in range(len(signs))]
            fields = [z[f"fields__{c}"] for c in range(n_chains)]
        self.ens.set_fields(fields, ctr)
        return bins

    def run(self, checkpoint: str | None = None, max_seconds: float | None = None) -> Result:
        """Warm up, then run the bins.  checkpoint: path of a file written after
        every bin; if it exists when the run starts, the run resumes from it (no
        warm-up).  max_seconds: stop after the first bin that ends past this
        wall-clock budget; the result covers the bins done (complete=False;
        with fewer than two bins its mean and error stay empty)."""
        t0 = time.monotonic()
        if checkpoint is not None and os.path.exists(checkpoint):
            bins = self._load(checkpoint)
        else:
            bins = []
            if self.warmup:
                self.ens.sweep(self.warmup, stats=False)
        while len(bins) < self.n_bins:
            bins.append(self._one_bin())
            if checkpoint is not None:
                self._save(checkpoint, bins)
            if max_seconds is not None and time.monotonic() - t0 >= max_seconds and len(bins) < self.n_bins:
                break
        return self._analyse(bins)

    def _analyse(self, bins) -> Result:
        res = Result(self.n_bins, self.sweeps_per_bin, 0.0, complete=len(bins) == self.n_bins)
        if (len(bins) - self.n_skip) // self.n_rebin < 2:
            return res

        def col(values):                       # per-bin values after n_skip and N_rebin
            return analysis.skip_and_rebin(np.array(values), self.n_skip, self.n_rebin)

        names = sorted({k for b, _ in bins for k in b if not k.startswith("_")})
        signs = col([s for _, s in bins])
        e_signs = col([b.get("_sign_energy", np.nan) for b, _ in bins])
        for k in names:
            data = col([b[k] for b, _ in bins])
            sg = e_signs if k in ("kin", "pot", "part", "ener") else signs
            res.mean[k], res.error[k] = analysis.jackknife(data, sg)
        if self.lattice is not None:
            a1, a2, L1, L2, n_orb, r_cells = self.lattice
            k = analysis.momenta(a1, a2, L1, L2)
            n_cells = k.shape[0]
            res.mean["k"] = k
            local = [(n_orb + 1) * a for a in range(n_orb)]                  # classes (d = 0, a, a)
            todo = []
            if self.corr is not None:
                gf = col([b["corr_gf"] for b, _ in bins])
                dens = gf[:, local] / n_cells                                   # sum_i n_ia / N_cell, sign-weighted
                todo += [(name, name + "_k", dens if name == "corr_nn" else None)
                         for name in ("corr_zz", "corr_nn", "corr_pm", "corr_gf")]
            if self.tau_corr is not None:
                g0 = col([b["gf_tau_r"] for b, _ in bins])[:, 0, :]            # tau = 0: sum_s G(0,0)_xx = 2 - n_x
                dens_t = 2.0 * signs[:, None] - g0[:, local] / n_cells
                todo += [(name, name[:-2] + "_k", dens_t if name == "nn_tau_r" else None)
                         for name in ("gf_tau_r", "szz_tau_r", "nn_tau_r")]
            for name, out, dens_b in todo:
                data = col([b[name] for b, _ in bins])
                want_cov = self.n_cov and name.endswith("_tau_r")
                r = analysis.obser_latt(data, signs, r_cells, a1, a2, k, n_cells, n_orb, O_sign=dens_b, cov=want_cov)
                res.mean[out], res.error[out] = r[0], r[1] + 1j * r[2]
                if want_cov:
                    res.cov[out] = r[3]
        if self.tau is not None or self.corr is not None or self.tau_corr is not None:
            res.mean_sign = float(signs.mean() / self._chains_total())  # per chain and sweep
        else:
            res.mean_sign = float(np.nanmean(e_signs))                 # per measurement
        return res
