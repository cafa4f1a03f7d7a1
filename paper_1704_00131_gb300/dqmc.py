"""ctypes binding of the C ABI in include/dqmc.h and include/dqmc_su2.h
(argument marshalling only).

Every step of the sweep runs in the CUDA kernels of libdqmc.so; this module
only packs numpy/torch arguments into the C structs and unpacks results.  It
raises if the library is missing: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from .workloads import ModelSpec

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libdqmc.so")

DQMC_OK, DQMC_EINVAL, DQMC_ENOMEM, DQMC_ECUDA, DQMC_EUNSTABLE, DQMC_ETIMEOUT, DQMC_ESTATE = range(7)
PREC = {"fp64": 0, "fp32": 1, "mixed": 2, "mixed_tc": 3}

EXPORTED = ["dqmc_init", "dqmc_sweep", "dqmc_greens", "dqmc_greens_tau", "dqmc_measure", "dqmc_measure_tau",
            "dqmc_measure_tau_corr", "dqmc_measure_corr", "dqmc_logdet_backward", "dqmc_energy_backward", "dqmc_get_fields",
            "dqmc_set_fields", "dqmc_green_fresh_noalloc", "dqmc_last_error", "dqmc_destroy",
            "dqmc_su2_init", "dqmc_su2_sweep", "dqmc_su2_greens", "dqmc_su2_measure", "dqmc_su2_measure_corr",
            "dqmc_su2_measure_tau", "dqmc_su2_greens_displaced",
            "dqmc_su2_get_fields",
            "dqmc_su2_set_fields", "dqmc_su2_last_error", "dqmc_su2_destroy"]


class DqmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"dqmc status {status}: {msg}")
        self.status = status


class ModelDesc(ctypes.Structure):
    _fields_ = [
        ("n_sites", ctypes.c_int32),
        ("n_flavors", ctypes.c_int32),
        ("hopping", ctypes.POINTER(ctypes.c_double)),
        ("n_vertices", ctypes.c_int32),
        ("vertex_site", ctypes.POINTER(ctypes.c_int32)),
        ("vertex_sign", ctypes.POINTER(ctypes.c_double)),
        ("U", ctypes.c_double),
        ("field_type", ctypes.c_int32),
        ("dtau", ctypes.c_double),
        ("L", ctypes.c_int32),
        ("n_wrap", ctypes.c_int32),
    ]


class RunOpts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("delay_k", ctypes.c_int32),
        ("measure", ctypes.c_int32),
        ("meas_first", ctypes.c_int32),
        ("meas_last", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("unstable_threshold", ctypes.c_double),
        ("spin_limit", ctypes.c_int64),
        ("tc_min_sites", ctypes.c_int32),
        ("dd_tile", ctypes.c_int32),
        ("test_stall", ctypes.c_int32),
        ("stab_svd", ctypes.c_int32),
    ]


class SweepStats(ctypes.Structure):
    _fields_ = [
        ("proposals", ctypes.c_int64),
        ("accepted", ctypes.c_int64),
        ("prec_green_mean", ctypes.c_double),
        ("prec_green_max", ctypes.c_double),
        ("prec_phase_max", ctypes.c_double),
        ("mean_sign", ctypes.c_double),
        ("ms_total", ctypes.c_float),
        ("ms_update", ctypes.c_float),
        ("ms_wrap", ctypes.c_float),
        ("ms_stab", ctypes.c_float),
        ("ms_measure", ctypes.c_float),
        ("ms_detail", ctypes.c_float * 8),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["ms_detail"] = list(self.ms_detail)
        return d


_lib = None


def lib_path() -> str:
    return _LIB_PATH


def load() -> ctypes.CDLL:
    """Load libdqmc.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with paper_1704_00131_gb300.build_ext.build()")
    L = ctypes.CDLL(_LIB_PATH)
    vp, i32, i64, u64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    L.dqmc_init.argtypes = [vp, i32, vp, i32, vp, vp, vp, ctypes.POINTER(vp)]
    L.dqmc_init.restype = ctypes.c_int
    L.dqmc_sweep.argtypes = [vp, i32, vp]
    L.dqmc_sweep.restype = ctypes.c_int
    L.dqmc_greens.argtypes = [vp, i32, i32, i32, vp, i32, vp, vp]
    L.dqmc_greens.restype = ctypes.c_int
    L.dqmc_greens_tau.argtypes = [vp, i32, i32, i32, vp, i32]
    L.dqmc_greens_tau.restype = ctypes.c_int
    L.dqmc_measure.argtypes = [vp, vp, vp, vp]
    L.dqmc_measure.restype = ctypes.c_int
    L.dqmc_measure_tau.argtypes = [vp, i32, vp, vp, vp, vp]
    L.dqmc_measure_tau.restype = ctypes.c_int
    L.dqmc_measure_tau_corr.argtypes = [vp, i32, vp, vp, vp, vp]
    L.dqmc_measure_tau_corr.restype = ctypes.c_int
    L.dqmc_measure_corr.argtypes = [vp, vp, vp, vp, vp]
    L.dqmc_measure_corr.restype = ctypes.c_int
    L.dqmc_logdet_backward.argtypes = [vp, i32, vp, i32, vp, vp, vp]
    L.dqmc_logdet_backward.restype = ctypes.c_int
    L.dqmc_energy_backward.argtypes = [vp, i32, vp, i32, vp, vp, vp]
    L.dqmc_energy_backward.restype = ctypes.c_int
    L.dqmc_get_fields.argtypes = [vp, vp, vp]
    L.dqmc_get_fields.restype = ctypes.c_int
    L.dqmc_set_fields.argtypes = [vp, vp, u64]
    L.dqmc_set_fields.restype = ctypes.c_int
    L.dqmc_last_error.argtypes = [vp]
    L.dqmc_last_error.restype = ctypes.c_char_p
    L.dqmc_destroy.argtypes = [vp]
    L.dqmc_destroy.restype = None
    L.dqmc_su2_init.argtypes = [vp, i32, vp, i32, vp, vp, vp, ctypes.POINTER(vp)]
    L.dqmc_su2_init.restype = ctypes.c_int
    L.dqmc_su2_sweep.argtypes = [vp, i32, vp]
    L.dqmc_su2_sweep.restype = ctypes.c_int
    L.dqmc_su2_greens.argtypes = [vp, i32, i32, vp, i32, vp, vp, vp]
    L.dqmc_su2_greens.restype = ctypes.c_int
    L.dqmc_su2_measure.argtypes = [vp, vp, vp, vp, i32]
    L.dqmc_su2_measure.restype = ctypes.c_int
    L.dqmc_su2_measure_tau.argtypes = [vp, i32, vp, vp]
    L.dqmc_su2_measure_tau.restype = ctypes.c_int
    L.dqmc_su2_greens_displaced.argtypes = [vp, i32, i32, vp, vp]
    L.dqmc_su2_greens_displaced.restype = ctypes.c_int
    L.dqmc_su2_measure_corr.argtypes = [vp, vp, vp, vp, vp]
    L.dqmc_su2_measure_corr.restype = ctypes.c_int
    L.dqmc_su2_get_fields.argtypes = [vp, vp, vp]
    L.dqmc_su2_get_fields.restype = ctypes.c_int
    L.dqmc_su2_set_fields.argtypes = [vp, vp, u64]
    L.dqmc_su2_set_fields.restype = ctypes.c_int
    L.dqmc_su2_last_error.argtypes = [vp]
    L.dqmc_su2_last_error.restype = ctypes.c_char_p
    L.dqmc_su2_destroy.argtypes = [vp]
    L.dqmc_su2_destroy.restype = None
    del i64, d
    _lib = L
    return L


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def szz_tau(obs: np.ndarray) -> np.ndarray:
    """sum_xy ph_x ph_y <S^z_x(tau) S^z_y(0)> per chain and tau from the two-flavor
    sums of Ensemble.measure_tau (flavor 0 up, flavor 1 down)."""
    m = obs[..., 0, 2] - obs[..., 1, 2]
    return (m * m[..., :1] + obs[..., 0, 1] + obs[..., 1, 1]) / 4.0


class Ensemble:
    """A set of Markov chains on one GPU (one dqmc_ctx)."""

    def __init__(self, models: list[ModelSpec], chain_model, fields=None, precision: str = "fp64",
                 delay_k: int = 16, seed: int = 0, measure: bool = False, meas_first: int = 0,
                 meas_last: int | None = None, unstable_threshold: float = 0.0, stream=None, spin_limit: int = 0,
                 tc_min_sites: int = 0, dd_tile: int = 0, test_stall: int = 0, stab_svd: bool = False):
        self._lib = load()
        self._h = ctypes.c_void_p()
        self.models = list(models)
        self.chain_model = np.ascontiguousarray(chain_model, dtype=np.int32)
        self.precision = precision
        self._keep = []
        descs = (ModelDesc * len(self.models))()
        for i, m in enumerate(self.models):
            H = np.ascontiguousarray(m.hopping, dtype=np.float64)
            vs = np.ascontiguousarray(m.vertex_site, dtype=np.int32)
            sg = np.ascontiguousarray(m.vertex_sign, dtype=np.float64)
            self._keep += [H, vs, sg]
            descs[i] = ModelDesc(m.N, H.shape[0], H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(vs),
                                 vs.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                 sg.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(m.U), int(m.field_type),
                                 float(m.dtau), int(m.L), int(m.n_wrap))
        self._descs = descs
        ml = max(m.L for m in self.models) if meas_last is None else meas_last
        self.opts = RunOpts(PREC[precision], int(delay_k), int(measure), int(meas_first), int(ml), int(seed),
                            float(unstable_threshold), int(spin_limit), int(tc_min_sites), int(dd_tile),
                            int(test_stall), int(bool(stab_svd)))
        fptr = None
        if fields is not None:
            packed = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.int8).ravel() for f in fields]))
            self._keep.append(packed)
            fptr = _p(packed)
        st_ptr = None
        if stream is not None:
            st_ptr = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        st = self._lib.dqmc_init(ctypes.cast(descs, ctypes.c_void_p), len(self.models), _p(self.chain_model),
                                 len(self.chain_model), fptr, ctypes.byref(self.opts), st_ptr, ctypes.byref(self._h))
        if st != DQMC_OK:
            msg = self._lib.dqmc_last_error(self._h).decode() if self._h else "dqmc_init failed"
            self.close()
            raise DqmcError(st, msg)

    # ------------------------------------------------------------------ helpers
    def _check(self, st: int):
        if st != DQMC_OK:
            raise DqmcError(st, self._lib.dqmc_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.dqmc_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_chains(self) -> int:
        return int(len(self.chain_model))

    def model_of(self, c: int) -> ModelSpec:
        return self.models[int(self.chain_model[c])]

    # --------------------------------------------------------------------- API
    def sweep(self, n: int = 1, stats: bool = True):
        if not stats:
            self._check(self._lib.dqmc_sweep(self._h, int(n), None))
            return None
        s = SweepStats()
        self._check(self._lib.dqmc_sweep(self._h, int(n), ctypes.byref(s)))
        return s.as_dict()

    def greens(self, chain: int, flavor: int, fresh: bool = False, out=None):
        """G^flavor(0) of a chain as a numpy array (or into a CUDA torch tensor `out`)."""
        if not 0 <= int(chain) < self.n_chains:
            raise DqmcError(DQMC_EINVAL, f"chain {chain} out of range")
        N = self.model_of(chain).N
        ld = ctypes.c_double()
        sg = ctypes.c_int32()
        if out is None:
            G = np.zeros((N, N))
            self._check(self._lib.dqmc_greens(self._h, chain, flavor, int(fresh), _p(G), 0, ctypes.byref(ld),
                                              ctypes.byref(sg)))
            return G, ld.value, sg.value
        self._check(self._lib.dqmc_greens(self._h, chain, flavor, int(fresh), ctypes.c_void_p(out.data_ptr()), 1,
                                          ctypes.byref(ld), ctypes.byref(sg)))
        return out, ld.value, sg.value

    def greens_tau(self, chain: int, flavor: int, tau: int, out=None):
        """G^flavor(tau) of a chain, wrapped in the working precision from the last
        stabilisation point tau0 <= tau with no accepted proposals (the drift probe
        of the precision monitor), as a numpy array (or into a CUDA torch tensor)."""
        if not 0 <= int(chain) < self.n_chains:
            raise DqmcError(DQMC_EINVAL, f"chain {chain} out of range")
        N = self.model_of(chain).N
        if out is None:
            G = np.zeros((N, N))
            self._check(self._lib.dqmc_greens_tau(self._h, int(chain), int(flavor), int(tau), _p(G), 0))
            return G
        self._check(self._lib.dqmc_greens_tau(self._h, int(chain), int(flavor), int(tau),
                                              ctypes.c_void_p(out.data_ptr()), 1))
        return out

    def measure(self):
        n = self.n_chains
        out = np.zeros((n, 4))
        ss = np.zeros(n)
        nm = np.zeros(n, dtype=np.int64)
        self._check(self._lib.dqmc_measure(self._h, _p(out), _p(ss), _p(nm)))
        return out, ss, nm

    def measure_tau(self, n_tau: int, site_phase=None):
        """Time-displaced sums of every chain's current configuration.

        Returns (obs, sign, prec): obs[c, tau, s] = (a, c, p) with
        a = sum_x G(tau,0)_xx, c = -sum_xy ph_x ph_y G(0,tau)_yx G(tau,0)_xy,
        p = sum_x ph_x (1 - G(tau,tau)_xx); sign[c, s] = sign of det(1 + B^s(beta,0));
        prec = (mean, max) of |wrapped - recomputed| time-displaced G ("Precision tau").
        site_phase: one array per model (or None for unit phases)."""
        nfl = max(m.hopping.shape[0] for m in self.models)
        obs = np.zeros((self.n_chains, int(n_tau) + 1, nfl, 3))
        sg = np.zeros((self.n_chains, nfl), dtype=np.int32)
        prec = np.zeros(2)
        ph = None
        if site_phase is not None:
            ph = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in site_phase]))
            if ph.size != sum(m.N for m in self.models):
                raise DqmcError(DQMC_EINVAL, "site_phase must hold one phase per site of every model")
        self._check(self._lib.dqmc_measure_tau(self._h, int(n_tau), None if ph is None else _p(ph), _p(obs), _p(sg),
                                               _p(prec)))
        return obs, sg, prec

    def measure_corr(self, pair_class, n_class):
        """Equal-time correlation sums per pair class of every chain's current
        configuration: out[c, k] = (S^z S^z, n n, S^+ S^-, sum_s c^+ c) summed over
        the pairs of class k; sign[c] = the configuration's sign.  pair_class and
        n_class: one entry per model (class map [N*N], number of classes)."""
        cls = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.int32).ravel() for a in pair_class]))
        nc = np.ascontiguousarray(n_class, dtype=np.int32)
        if cls.size != sum(m.N * m.N for m in self.models) or nc.size != len(self.models):
            raise DqmcError(DQMC_EINVAL, "one class map [N*N] and one class count per model")
        out = np.zeros((self.n_chains, int(nc.max()), 4))
        sg = np.zeros(self.n_chains, dtype=np.int32)
        self._check(self._lib.dqmc_measure_corr(self._h, _p(cls), _p(nc), _p(out), _p(sg)))
        return out, sg

    def measure_tau_corr(self, n_tau: int, pair_class, n_class):
        """Time-displaced correlation sums per pair class of every chain's current
        configuration: out[c, tau, k] = (sum_s <c_xs(tau) c^+_ys(0)>, <S^z_x(tau) S^z_y(0)>,
        <n_x(tau) n_y(0)>) summed over the pairs (x, y) of class k; sign[c] = the
        configuration's sign.  pair_class and n_class: one entry per model."""
        cls = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.int32).ravel() for a in pair_class]))
        nc = np.ascontiguousarray(n_class, dtype=np.int32)
        if cls.size != sum(m.N * m.N for m in self.models) or nc.size != len(self.models):
            raise DqmcError(DQMC_EINVAL, "one class map [N*N] and one class count per model")
        out = np.zeros((self.n_chains, int(n_tau) + 1, int(nc.max()), 3))
        sg = np.zeros(self.n_chains, dtype=np.int32)
        self._check(self._lib.dqmc_measure_tau_corr(self._h, int(n_tau), _p(cls), _p(nc), _p(out), _p(sg)))
        return out, sg

    def get_fields(self):
        sizes = [self.model_of(c).L * self.model_of(c).n_vertices for c in range(self.n_chains)]
        buf = np.zeros(sum(sizes), dtype=np.int8)
        ctr = ctypes.c_uint64()
        self._check(self._lib.dqmc_get_fields(self._h, _p(buf), ctypes.byref(ctr)))
        out, off = [], 0
        for c, sz in enumerate(sizes):
            m = self.model_of(c)
            out.append(buf[off:off + sz].reshape(m.L, m.n_vertices).copy())
            off += sz
        return out, ctr.value

    def set_fields(self, fields, rng_counter: int):
        packed = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.int8).ravel() for f in fields]))
        self._check(self._lib.dqmc_set_fields(self._h, _p(packed), int(rng_counter)))

    def logdet_backward(self, model_index: int, fields: np.ndarray):
        """Per configuration and flavor: log|det(1+B(beta,0))|, d/dK (symmetric pairs), d/dU."""
        m = self.models[model_index]
        f = np.ascontiguousarray(fields, dtype=np.int8)
        if f.ndim == 2:
            f = f[None]
        n_cfg = f.shape[0]
        nfl = m.hopping.shape[0]
        ldv = np.zeros((n_cfg, nfl))
        gK = np.zeros((n_cfg, nfl, m.N, m.N))
        gU = np.zeros((n_cfg, nfl))
        self._check(self._lib.dqmc_logdet_backward(self._h, int(model_index), _p(f), n_cfg, _p(ldv), _p(gK), _p(gU)))
        return ldv, gK, gU

    def energy_backward(self, model_index: int, fields: np.ndarray):
        """Per configuration: (Kin, Pot, Part, Ener), dEner/dK^s (symmetric pairs) and dEner/dU."""
        m = self.models[model_index]
        f = np.ascontiguousarray(fields, dtype=np.int8)
        if f.ndim == 2:
            f = f[None]
        n_cfg = f.shape[0]
        nfl = m.hopping.shape[0]
        e = np.zeros((n_cfg, 4))
        gK = np.zeros((n_cfg, nfl, m.N, m.N))
        gU = np.zeros(n_cfg)
        self._check(self._lib.dqmc_energy_backward(self._h, int(model_index), _p(f), n_cfg, _p(e), _p(gK), _p(gU)))
        return e, gK, gU


# ---------------------------------------------------------------------------
# SU(2) charge decoupling with complex coupling (include/dqmc_su2.h)
# ---------------------------------------------------------------------------
class Su2ModelDesc(ctypes.Structure):
    _fields_ = [
        ("n_sites", ctypes.c_int32),
        ("hopping", ctypes.POINTER(ctypes.c_double)),
        ("U", ctypes.c_double),
        ("dtau", ctypes.c_double),
        ("L", ctypes.c_int32),
        ("n_wrap", ctypes.c_int32),
        ("n_bonds", ctypes.c_int32),
        ("bond_sites", ctypes.POINTER(ctypes.c_int32)),
        ("xi", ctypes.c_double),
        ("h", ctypes.c_double),
        ("J", ctypes.c_double),
        ("n_pairs", ctypes.c_int32),
        ("pairs", ctypes.POINTER(ctypes.c_int32)),
    ]


class Su2Opts(ctypes.Structure):
    _fields_ = [
        ("measure", ctypes.c_int32),
        ("meas_first", ctypes.c_int32),
        ("meas_last", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("unstable_threshold", ctypes.c_double),
    ]


class Su2SweepStats(ctypes.Structure):
    _fields_ = [
        ("proposals", ctypes.c_int64),
        ("accepted", ctypes.c_int64),
        ("prec_green_mean", ctypes.c_double),
        ("prec_green_max", ctypes.c_double),
        ("prec_phase_max", ctypes.c_double),
        ("mean_sign", ctypes.c_double),
        ("ms_total", ctypes.c_float),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


@dataclass
class Su2Model:
    """One lattice of the SU(2) Hubbard model: hopping K [N, N] (-mu on the
    diagonal), U, dtau, L slices, stabilisation interval n_wrap; optionally
    Ising spins on `bonds` [(i, j), ...] coupled to their hopping by xi, with a
    transverse field h and a coupling J between the bond `pairs` [(b, b'), ...]
    (the Hubbard-Ising model)."""
    hopping: np.ndarray
    U: float
    dtau: float
    L: int
    n_wrap: int
    bonds: tuple = ()
    xi: float = 0.0
    h: float = 0.0
    J: float = 0.0
    pairs: tuple = ()

    @property
    def N(self) -> int:
        return int(self.hopping.shape[0])

    @property
    def n_bonds(self) -> int:
        return len(self.bonds)

    @property
    def MV(self) -> int:
        return self.N + self.n_bonds


class Su2Ensemble:
    """Markov chains of the SU(2) decoupling on one GPU (one dqmc_su2_ctx)."""

    def __init__(self, models: list[Su2Model], chain_model, fields=None, seed: int = 0, measure: bool = False,
                 meas_first: int = 0, meas_last: int | None = None, unstable_threshold: float = 0.0, stream=None):
        self._lib = load()
        self._h = ctypes.c_void_p()
        self.models = list(models)
        self.chain_model = np.ascontiguousarray(chain_model, dtype=np.int32)
        self._keep = []
        descs = (Su2ModelDesc * len(self.models))()
        i32p = ctypes.POINTER(ctypes.c_int32)
        for i, m in enumerate(self.models):
            H = np.ascontiguousarray(m.hopping, dtype=np.float64)
            bs = np.ascontiguousarray(np.asarray(m.bonds, dtype=np.int32).reshape(-1, 2))
            ps = np.ascontiguousarray(np.asarray(m.pairs, dtype=np.int32).reshape(-1, 2))
            self._keep += [H, bs, ps]
            descs[i] = Su2ModelDesc(m.N, H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(m.U),
                                    float(m.dtau), int(m.L), int(m.n_wrap), len(bs), bs.ctypes.data_as(i32p),
                                    float(m.xi), float(m.h), float(m.J), len(ps), ps.ctypes.data_as(i32p))
        self._descs = descs
        ml = max(m.L for m in self.models) if meas_last is None else meas_last
        self.opts = Su2Opts(int(measure), int(meas_first), int(ml), int(seed), float(unstable_threshold))
        fptr = None
        if fields is not None:
            packed = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.int8).ravel() for f in fields]))
            self._keep.append(packed)
            fptr = _p(packed)
        st_ptr = None
        if stream is not None:
            st_ptr = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        st = self._lib.dqmc_su2_init(ctypes.cast(descs, ctypes.c_void_p), len(self.models), _p(self.chain_model),
                                     len(self.chain_model), fptr, ctypes.byref(self.opts), st_ptr,
                                     ctypes.byref(self._h))
        if st != DQMC_OK:
            msg = self._lib.dqmc_su2_last_error(self._h).decode() if self._h.value else "init failed"
            self.close()
            raise DqmcError(st, msg)

    def _check(self, st: int):
        if st != DQMC_OK:
            raise DqmcError(st, self._lib.dqmc_su2_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.dqmc_su2_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_chains(self) -> int:
        return int(len(self.chain_model))

    def model_of(self, c: int) -> Su2Model:
        return self.models[int(self.chain_model[c])]

    def sweep(self, n: int = 1) -> dict:
        s = Su2SweepStats()
        self._check(self._lib.dqmc_su2_sweep(self._h, int(n), ctypes.byref(s)))
        return s.as_dict()

    def greens(self, chain: int, fresh: bool = False):
        """(G(0) complex [N, N], log|det(1+B)|, arg det(1+B), phase P complex) of a chain."""
        N = self.model_of(chain).N
        G = np.zeros((N, N, 2))
        la, ar = ctypes.c_double(), ctypes.c_double()
        ph = np.zeros(2)
        self._check(self._lib.dqmc_su2_greens(self._h, int(chain), int(fresh), _p(G), 0, ctypes.byref(la),
                                              ctypes.byref(ar), _p(ph)))
        return G[..., 0] + 1j * G[..., 1], la.value, ar.value, complex(ph[0], ph[1])

    def measure(self, reset: bool = False):
        """(complex [n_chains, 5] reweighted sums of Kin, Pot, Part, Ener and the bond
        spins' (sum_b s_b)^2 / n_bonds; sign sums; counts)."""
        out = np.zeros((self.n_chains, 5, 2))
        sg = np.zeros(self.n_chains)
        nm = np.zeros(self.n_chains, dtype=np.int64)
        self._check(self._lib.dqmc_su2_measure(self._h, _p(out), _p(sg), _p(nm), int(reset)))
        return out[..., 0] + 1j * out[..., 1], sg, nm

    def measure_tau(self, n_tau: int):
        """(complex [n_chains, n_tau + 1] traces of G(tau,0); (mean, max) of Precision tau)."""
        out = np.zeros((self.n_chains, int(n_tau) + 1, 2))
        pt = np.zeros(2)
        self._check(self._lib.dqmc_su2_measure_tau(self._h, int(n_tau), _p(out), _p(pt)))
        return out[..., 0] + 1j * out[..., 1], (float(pt[0]), float(pt[1]))

    def greens_displaced(self, chain: int, tau: int):
        """(G(tau,0), G(0,tau)) of a chain, complex [N, N] each."""
        N = self.model_of(chain).N
        a = np.zeros((N, N, 2))
        b = np.zeros((N, N, 2))
        self._check(self._lib.dqmc_su2_greens_displaced(self._h, int(chain), int(tau), _p(a), _p(b)))
        return a[..., 0] + 1j * a[..., 1], b[..., 0] + 1j * b[..., 1]

    def measure_corr(self, pair_class, n_class):
        """Equal-time correlations per pair class of every chain's current G(0):
        (complex [n_chains, max n_class, 4] sums of S^z S^z, n n, S^+ S^-, c^+ c;
        complex phase P per chain).  pair_class: one [N, N] int array per model."""
        cls = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.int32).ravel() for c in pair_class]))
        nc = np.ascontiguousarray(n_class, dtype=np.int32)
        out = np.zeros((self.n_chains, int(nc.max()), 4, 2))
        ph = np.zeros((self.n_chains, 2))
        self._check(self._lib.dqmc_su2_measure_corr(self._h, _p(cls), _p(nc), _p(out), _p(ph)))
        return out[..., 0] + 1j * out[..., 1], ph[:, 0] + 1j * ph[:, 1]

    def get_fields(self):
        total = sum(self.model_of(c).L * self.model_of(c).MV for c in range(self.n_chains))
        buf = np.zeros(total, dtype=np.int8)
        ctr = ctypes.c_uint64()
        self._check(self._lib.dqmc_su2_get_fields(self._h, _p(buf), ctypes.byref(ctr)))
        out, off = [], 0
        for c in range(self.n_chains):
            m = self.model_of(c)
            out.append(buf[off:off + m.L * m.MV].reshape(m.L, m.MV).copy())
            off += m.L * m.MV
        return out, ctr.value

    def set_fields(self, fields, sweep_counter: int = 0):
        packed = np.ascontiguousarray(np.concatenate([np.asarray(f, dtype=np.int8).ravel() for f in fields]))
        self._check(self._lib.dqmc_su2_set_fields(self._h, _p(packed), int(sweep_counter)))
