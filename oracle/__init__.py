"""FP64 CPU oracle of the BSS/DQMC sweep (ALF 1.0 documentation, arXiv:1704.00131).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import this package.  The CUDA library of
``paper_1704_00131_gb300`` never imports, links or calls it, and the two share no
code: the oracle is plain C (``dqmc_oracle.c``) built with gcc, loaded here with
ctypes, and every array crossing this wrapper is a plain numpy array.

Parity unpinned: nothing here is unpinned; see the tests under ``tests/`` that
pin each routine (closed forms, exact diagonalisation, symmetries, brute force).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dqmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

FIELD_ISING = 1
FIELD_HS4 = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable C99, no architecture flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Model(ctypes.Structure):
    _fields_ = [
        ("n_sites", ctypes.c_int32),
        ("n_flavors", ctypes.c_int32),
        ("n_vertices", ctypes.c_int32),
        ("field_type", ctypes.c_int32),
        ("L", ctypes.c_int32),
        ("n_wrap", ctypes.c_int32),
        ("dtau", ctypes.c_double),
        ("U", ctypes.c_double),
        ("hopping", ctypes.POINTER(ctypes.c_double)),
        ("vertex_site", ctypes.POINTER(ctypes.c_int32)),
        ("vertex_sign", ctypes.POINTER(ctypes.c_double)),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("proposals", ctypes.c_int64),
        ("accepted", ctypes.c_int64),
        ("prec_green_mean", ctypes.c_double),
        ("prec_green_max", ctypes.c_double),
        ("prec_phase_max", ctypes.c_double),
        ("mean_sign", ctypes.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # DQMC_ORACLE_LIB: a prebuilt oracle library to load instead (the pin
        # tests load builds with planted mistakes this way and must fail)
        _lib = ctypes.CDLL(os.environ.get("DQMC_ORACLE_LIB") or build())
        d, i32, u32, u64, vp = ctypes.c_double, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p
        _lib.orc_philox4x32_10.argtypes = [vp, vp, vp]
        _lib.orc_u01.argtypes = [u32, u32]
        _lib.orc_u01.restype = d
        _lib.orc_init_fields.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u64, u32, vp]
        _lib.orc_field_coupling.argtypes = [ctypes.c_int, d, d, ctypes.c_int]
        _lib.orc_field_coupling.restype = d
        _lib.orc_field_gamma.argtypes = [ctypes.c_int, ctypes.c_int]
        _lib.orc_field_gamma.restype = d
        _lib.orc_ising_lambda.argtypes = [d, d]
        _lib.orc_ising_lambda.restype = d
        _lib.orc_eig_sym.argtypes = [ctypes.c_int, vp, vp, vp]
        _lib.orc_expm_sym.argtypes = [ctypes.c_int, vp, d, vp]
        _lib.orc_logdet.argtypes = [ctypes.c_int, vp, vp, vp]
        _lib.orc_green_plain.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        _lib.orc_green_udv.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        _lib.orc_green_udv_svd.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp, vp]
        _lib.orc_energy.argtypes = [vp, vp, vp]
        _lib.orc_chain_new.argtypes = [vp, vp, u64, u32, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib.orc_chain_new.restype = vp
        _lib.orc_chain_free.argtypes = [vp]
        _lib.orc_chain_sweep.argtypes = [vp, ctypes.c_int, vp]
        _lib.orc_chain_green.argtypes = [vp, ctypes.c_int, vp]
        _lib.orc_chain_fields.argtypes = [vp, vp, vp, vp]
        _lib.orc_chain_measure.argtypes = [vp, vp, vp, vp]
        _lib.orc_logdet_grad.argtypes = [vp, vp, vp, vp, vp, vp]
        _lib.orc_green_displaced.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, vp, vp]
        _lib.orc_energy_grad.argtypes = [vp, vp, vp, vp, vp]
        _lib.orc_tau_observables.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp]
        _lib.orc_correlations.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int, vp]
        _lib.orc_su2_plain.argtypes = [ctypes.c_int, vp, d, d, ctypes.c_int, vp, vp, vp, vp, vp, vp]
        _lib.orc_su2_sweep.argtypes = [ctypes.c_int, vp, d, d, ctypes.c_int, vp, u64, u32, u64, vp, vp, vp]
        _lib.orc_hubbard_ising_plain.argtypes = [ctypes.c_int, vp, ctypes.c_int, vp, vp, d, d, d, ctypes.c_int, vp, vp, vp,
                                                  vp, vp, vp, vp]
        _lib.orc_ising_bond_logweight.argtypes = [ctypes.c_int, ctypes.c_int, vp, d, d, d, ctypes.c_int, vp, vp]
        _lib.orc_hubbard_ising_green_at.argtypes = [ctypes.c_int, vp, ctypes.c_int, vp, vp, d, d, d, ctypes.c_int, vp,
                                                     vp, ctypes.c_int, ctypes.c_int, vp]
        _lib.orc_bond_rank2_update.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, vp]
        _lib.orc_hubbard_ising_sweep.argtypes = [ctypes.c_int, vp, ctypes.c_int, vp, vp, d, d, d, ctypes.c_int, vp, d, d,
                                                 ctypes.c_int, vp, vp, u64, u32, u64, vp, vp, vp]
        _lib.orc_tau_correlations.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int, vp]
        _lib.orc_hubbard_ising_green_udv.argtypes = [ctypes.c_int, vp, ctypes.c_int, vp, vp, d, d, d, ctypes.c_int,
                                                      ctypes.c_int, vp, vp, ctypes.c_int, vp, vp, vp]
        _lib.orc_su2_correlations.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int, vp]
        _lib.orc_su2_green_udv.argtypes = [ctypes.c_int, vp, d, d, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp]
        _lib.orc_su2_green_displaced.argtypes = [ctypes.c_int, vp, d, d, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int,
                                                 vp, vp]
        del i32
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Model:
    """A Hubbard-type model: hopping per flavor, single-site vertices, one field type."""

    hopping: np.ndarray          # [n_flavors, N, N] float64, symmetric, includes -mu
    vertex_site: np.ndarray      # [M_V] int32
    vertex_sign: np.ndarray      # [n_flavors, M_V] float64 (sigma_s)
    U: float
    dtau: float
    L: int
    n_wrap: int
    field_type: int = FIELD_ISING

    def __post_init__(self):
        self.hopping = np.ascontiguousarray(self.hopping, dtype=np.float64)
        if self.hopping.ndim == 2:
            self.hopping = np.ascontiguousarray(np.stack([self.hopping, self.hopping]))
        self.vertex_site = np.ascontiguousarray(self.vertex_site, dtype=np.int32)
        self.vertex_sign = np.ascontiguousarray(self.vertex_sign, dtype=np.float64)
        self._c = _Model(
            self.N, self.n_flavors, self.n_vertices, int(self.field_type), int(self.L), int(self.n_wrap),
            float(self.dtau), float(self.U),
            self.hopping.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            self.vertex_site.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            self.vertex_sign.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        )

    @property
    def N(self) -> int:
        return int(self.hopping.shape[-1])

    @property
    def n_flavors(self) -> int:
        return int(self.hopping.shape[0])

    @property
    def n_vertices(self) -> int:
        return int(self.vertex_site.shape[0])

    def cref(self):
        return ctypes.byref(self._c)


def _check(st: int, what: str):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(hi: int, lo: int) -> float:
    return lib().orc_u01(hi, lo)


def init_fields(field_type: int, L: int, MV: int, seed: int, chain: int) -> np.ndarray:
    f = np.zeros((L, MV), dtype=np.int8)
    lib().orc_init_fields(field_type, L, MV, seed, chain, _ptr(f))
    return f


def field_coupling(field_type: int, dtau: float, U: float, f: int) -> float:
    return lib().orc_field_coupling(field_type, dtau, U, f)


def field_gamma(field_type: int, f: int) -> float:
    return lib().orc_field_gamma(field_type, f)


def ising_lambda(dtau: float, U: float) -> float:
    return lib().orc_ising_lambda(dtau, U)


def eig_sym(A: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n))
    lib().orc_eig_sym(n, _ptr(A), _ptr(w), _ptr(V))
    return w, V


def expm_sym(K: np.ndarray, t: float) -> np.ndarray:
    K = np.ascontiguousarray(K, dtype=np.float64)
    E = np.zeros_like(K)
    lib().orc_expm_sym(K.shape[0], _ptr(K), t, _ptr(E))
    return E


def logdet(A: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.float64)
    ld = ctypes.c_double()
    sg = ctypes.c_int()
    _check(lib().orc_logdet(A.shape[0], _ptr(A), ctypes.byref(ld), ctypes.byref(sg)), "logdet")
    return ld.value, sg.value


def _green(fn, model: Model, fields: np.ndarray, flavor: int, tau: int):
    f = np.ascontiguousarray(fields, dtype=np.int8)
    G = np.zeros((model.N, model.N))
    ld = ctypes.c_double()
    sg = ctypes.c_int()
    _check(fn(model.cref(), _ptr(f), flavor, tau, _ptr(G), ctypes.byref(ld), ctypes.byref(sg)), "green")
    return G, ld.value, sg.value


def green_plain(model: Model, fields: np.ndarray, flavor: int, tau: int = 0):
    """G(tau) = (1 + B(tau,0) B(beta,tau))^-1 by the plain product and LU."""
    return _green(lib().orc_green_plain, model, fields, flavor, tau)


def green_udv(model: Model, fields: np.ndarray, flavor: int, tau: int = 0):
    """G(tau) through the QR-stabilised UDV chains (chunks of n_wrap slices)."""
    return _green(lib().orc_green_udv, model, fields, flavor, tau)


def green_udv_svd(model: Model, fields: np.ndarray, flavor: int, tau: int = 0):
    """G(tau) through UDV chains decomposed by one-sided Jacobi SVD (the SVD
    stabilisation option) instead of the pivoted QR."""
    return _green(lib().orc_green_udv_svd, model, fields, flavor, tau)


def energy(model: Model, G: np.ndarray) -> np.ndarray:
    """(Kin, Pot, Part, Ener) of one configuration from G[n_flavors, N, N]."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    out = np.zeros(4)
    _check(lib().orc_energy(model.cref(), _ptr(G), _ptr(out)), "energy")
    return out


class Chain:
    """One Markov chain of the oracle (plain Sherman-Morrison updates, FP64)."""

    def __init__(self, model: Model, fields=None, seed: int = 0, chain: int = 0, measure: bool = False,
                 meas_first: int = 0, meas_last: int | None = None):
        self.model = model
        self._fields_in = None if fields is None else np.ascontiguousarray(fields, dtype=np.int8)
        ml = model.L if meas_last is None else meas_last
        self._h = lib().orc_chain_new(model.cref(), None if self._fields_in is None else _ptr(self._fields_in),
                                      seed, chain, int(measure), meas_first, ml)
        if not self._h:
            raise RuntimeError("oracle chain creation failed")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_chain_free(h)
            self._h = None

    def sweep(self, n: int = 1) -> Stats:
        st = Stats()
        _check(lib().orc_chain_sweep(self._h, n, ctypes.byref(st)), "sweep")
        return st

    def green(self, flavor: int) -> np.ndarray:
        G = np.zeros((self.model.N, self.model.N))
        _check(lib().orc_chain_green(self._h, flavor, _ptr(G)), "chain_green")
        return G

    def fields(self):
        f = np.zeros((self.model.L, self.model.n_vertices), dtype=np.int8)
        sw = ctypes.c_uint64()
        sg = ctypes.c_int()
        _check(lib().orc_chain_fields(self._h, _ptr(f), ctypes.byref(sw), ctypes.byref(sg)), "fields")
        return f, sw.value, sg.value

    def measure(self):
        out = np.zeros(4)
        ss = ctypes.c_double()
        nm = ctypes.c_int64()
        _check(lib().orc_chain_measure(self._h, _ptr(out), ctypes.byref(ss), ctypes.byref(nm)), "measure")
        return out, ss.value, nm.value


def logdet_grad(model: Model, fields: np.ndarray):
    """Per flavor: log|det(1+B(beta,0))|, its sign, d/dK (symmetric pairs) and d/dU."""
    f = np.ascontiguousarray(fields, dtype=np.int8)
    nfl, N = model.n_flavors, model.N
    ld = np.zeros(nfl)
    sg = np.zeros(nfl, dtype=np.int32)
    gK = np.zeros((nfl, N, N))
    gU = np.zeros(nfl)
    _check(lib().orc_logdet_grad(model.cref(), _ptr(f), _ptr(ld), _ptr(sg), _ptr(gK), _ptr(gU)), "logdet_grad")
    return ld, sg, gK, gU


def green_displaced(model: Model, fields: np.ndarray, flavor: int, tau: int):
    """G(tau,0) and G(0,tau) through the UDV chains."""
    f = np.ascontiguousarray(fields, dtype=np.int8)
    Gt0 = np.zeros((model.N, model.N))
    G0t = np.zeros((model.N, model.N))
    _check(lib().orc_green_displaced(model.cref(), _ptr(f), flavor, tau, _ptr(Gt0), _ptr(G0t)), "green_displaced")
    return Gt0, G0t


def tau_observables(model: Model, fields: np.ndarray, n_tau: int, phase=None):
    """Per displacement tau = 0..n_tau and flavor s: (a_s, c_s, p_s) =
    (sum_x G(tau,0)_xx, -sum_xy ph_x ph_y G(0,tau)_yx G(tau,0)_xy, sum_x ph_x (1 - G(tau,tau)_xx)),
    every Green function from scratch; returns (out[n_tau+1, nfl, 3], signs[nfl])."""
    f = np.ascontiguousarray(fields, dtype=np.int8)
    out = np.zeros((n_tau + 1, model.n_flavors, 3))
    sg = np.zeros(model.n_flavors, dtype=np.int32)
    ph = None if phase is None else np.ascontiguousarray(phase, dtype=np.float64)
    _check(lib().orc_tau_observables(model.cref(), _ptr(f), n_tau, None if ph is None else _ptr(ph), _ptr(out),
                                     _ptr(sg)), "tau_observables")
    return out, sg


def tau_correlations(model: Model, fields: np.ndarray, n_tau: int, pair_class: np.ndarray, n_class: int):
    """Per displacement tau = 0..n_tau and pair class: sums of sum_s <c_xs(tau) c^+_ys(0)>,
    <S^z_x(tau) S^z_y(0)> and <n_x(tau) n_y(0)> of one configuration; returns [n_tau+1, n_class, 3]."""
    f = np.ascontiguousarray(fields, dtype=np.int8)
    cls = np.ascontiguousarray(pair_class, dtype=np.int32)
    out = np.zeros((n_tau + 1, n_class, 3))
    _check(lib().orc_tau_correlations(model.cref(), _ptr(f), int(n_tau), _ptr(cls), int(n_class), _ptr(out)),
           "tau_correlations")
    return out


def correlations(G: np.ndarray, pair_class: np.ndarray, n_class: int) -> np.ndarray:
    """Equal-time (S^z S^z, n n, S^+ S^-, sum_s c^+ c) sums per pair class of one
    configuration from its two-flavor Green functions G[2, N, N]; returns [n_class, 4]."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    N = G.shape[-1]
    cls = np.ascontiguousarray(pair_class, dtype=np.int32).reshape(N, N)
    out = np.zeros((n_class, 4))
    _check(lib().orc_correlations(N, _ptr(G), _ptr(cls), int(n_class), _ptr(out)), "correlations")
    return out


def su2_plain(K: np.ndarray, dtau: float, U: float, fields: np.ndarray):
    """SU(2) charge decoupling with complex coupling, plain product (small beta):
    returns (G complex [N, N], log|det(1+B)|, arg det(1+B), phase -g sum eta,
    Kin + i.., Pot + i.. of the configuration)."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    N = K.shape[0]
    f = np.ascontiguousarray(fields, dtype=np.int8)
    L = f.size // N
    G = np.zeros((N, N, 2))
    la, ar, ph = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    e = np.zeros(4)
    _check(lib().orc_su2_plain(N, _ptr(K), float(dtau), float(U), L, _ptr(f), _ptr(G), ctypes.byref(la),
                               ctypes.byref(ar), ctypes.byref(ph), _ptr(e)), "su2_plain")
    return G[..., 0] + 1j * G[..., 1], la.value, ar.value, ph.value, complex(e[0], e[1]), complex(e[2], e[3])


def su2_correlations(G: np.ndarray, pair_class: np.ndarray, n_class: int) -> np.ndarray:
    """Equal-time (S^z S^z, n n, S^+ S^-, sum_s c^+ c) sums per pair class of one
    configuration of the SU(2) decoupling from its complex G [N, N] (both colors);
    returns complex [n_class, 4]."""
    N = G.shape[0]
    Gi = np.ascontiguousarray(np.stack([G.real, G.imag], axis=-1), dtype=np.float64)
    cls = np.ascontiguousarray(pair_class, dtype=np.int32)
    out = np.zeros((n_class, 4, 2))
    _check(lib().orc_su2_correlations(N, _ptr(Gi), _ptr(cls), int(n_class), _ptr(out)), "su2_correlations")
    return out[..., 0] + 1j * out[..., 1]


def su2_green_displaced(K: np.ndarray, dtau: float, U: float, n_wrap: int, fields: np.ndarray, tau: int):
    """G(tau,0) and G(0,tau) (complex [N, N]) of one color of the SU(2)
    decoupling through the complex UDV chains."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    N = K.shape[0]
    f = np.ascontiguousarray(fields, dtype=np.int8)
    L = f.size // N
    Gt0 = np.zeros((N, N, 2))
    G0t = np.zeros((N, N, 2))
    _check(lib().orc_su2_green_displaced(N, _ptr(K), float(dtau), float(U), L, int(n_wrap), _ptr(f), int(tau),
                                         _ptr(Gt0), _ptr(G0t)), "su2_green_displaced")
    return Gt0[..., 0] + 1j * Gt0[..., 1], G0t[..., 0] + 1j * G0t[..., 1]


def su2_green_udv(K: np.ndarray, dtau: float, U: float, n_wrap: int, fields: np.ndarray, tau: int = 0):
    """G(tau) of one color of the SU(2) decoupling through the complex UDV chains:
    (G complex [N, N], log|det(1 + B(beta,0))|, arg det(1 + B(beta,0)))."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    N = K.shape[0]
    f = np.ascontiguousarray(fields, dtype=np.int8)
    L = f.size // N
    G = np.zeros((N, N, 2))
    la, ar = ctypes.c_double(), ctypes.c_double()
    _check(lib().orc_su2_green_udv(N, _ptr(K), float(dtau), float(U), L, int(n_wrap), _ptr(f), int(tau), _ptr(G),
                                   ctypes.byref(la), ctypes.byref(ar)), "su2_green_udv")
    return G[..., 0] + 1j * G[..., 1], la.value, ar.value


def hubbard_ising_plain(T: np.ndarray, bonds, xi: float, dtau: float, U: float, hs: np.ndarray, ising: np.ndarray):
    """SU(2) Hubbard model with an Ising field on bonds coupling to the hopping, on
    fixed HS fields hs[L, N] and Ising spins ising[L, n_bonds]: (G complex,
    log|det(1+B)|, arg det(1+B), HS phase, Kin complex) of one color."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    N = T.shape[0]
    b = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
    bi, bj = np.ascontiguousarray(b[:, 0]), np.ascontiguousarray(b[:, 1])
    f = np.ascontiguousarray(hs, dtype=np.int8)
    z = np.ascontiguousarray(ising, dtype=np.int8)
    L = f.size // N
    G = np.zeros((N, N, 2))
    la, ar, ph = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    kin = np.zeros(2)
    _check(lib().orc_hubbard_ising_plain(N, _ptr(T), len(bi), _ptr(bi), _ptr(bj), float(xi), float(dtau), float(U), L,
                                         _ptr(f), _ptr(z), _ptr(G), ctypes.byref(la), ctypes.byref(ar),
                                         ctypes.byref(ph), _ptr(kin)), "hubbard_ising_plain")
    return G[..., 0] + 1j * G[..., 1], la.value, ar.value, ph.value, complex(kin[0], kin[1])


def ising_bond_logweight(ising: np.ndarray, dtau: float, h: float, J: float, pairs) -> float:
    """log of the imaginary-time weight of the bond Ising spins ising[L, n_bonds]."""
    z = np.ascontiguousarray(ising, dtype=np.int8)
    L, nb = z.shape
    p = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    lw = ctypes.c_double()
    _check(lib().orc_ising_bond_logweight(nb, L, _ptr(z), float(dtau), float(h), float(J), len(p),
                                          _ptr(p) if len(p) else None, ctypes.byref(lw)), "ising_bond_logweight")
    return lw.value


def _bond_arrays(bonds):
    b = np.ascontiguousarray(bonds, dtype=np.int32).reshape(-1, 2)
    return np.ascontiguousarray(b[:, 0]), np.ascontiguousarray(b[:, 1])


def hubbard_ising_green_at(T: np.ndarray, bonds, xi: float, dtau: float, U: float, hs: np.ndarray,
                           ising: np.ndarray, tau: int, part: int) -> np.ndarray:
    """Green function (complex [N, N]) seen by the factor (tau, part) of the bond
    model: part 0 = the HS factor of slice tau, 1..n_bonds = bonds n_bonds-1..0,
    n_bonds+1 = exp(-dtau T)."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    N = T.shape[0]
    bi, bj = _bond_arrays(bonds)
    f = np.ascontiguousarray(hs, dtype=np.int8)
    z = np.ascontiguousarray(ising, dtype=np.int8)
    G = np.zeros((N, N, 2))
    _check(lib().orc_hubbard_ising_green_at(N, _ptr(T), len(bi), _ptr(bi), _ptr(bj), float(xi), float(dtau),
                                            float(U), f.size // N, _ptr(f), _ptr(z), int(tau), int(part), _ptr(G)),
           "hubbard_ising_green_at")
    return G[..., 0] + 1j * G[..., 1]


def hubbard_ising_green_udv(T: np.ndarray, bonds, xi: float, dtau: float, U: float, n_wrap: int, hs: np.ndarray,
                            ising: np.ndarray, tau: int = 0):
    """G(tau) of one color of the bond model through the complex UDV chains:
    (G complex [N, N], log|det(1 + B(beta,0))|, arg det(1 + B(beta,0)))."""
    T = np.ascontiguousarray(T, dtype=np.float64)
    N = T.shape[0]
    bi, bj = _bond_arrays(bonds)
    f = np.ascontiguousarray(hs, dtype=np.int8)
    z = np.ascontiguousarray(ising, dtype=np.int8)
    G = np.zeros((N, N, 2))
    la, ar = ctypes.c_double(), ctypes.c_double()
    _check(lib().orc_hubbard_ising_green_udv(N, _ptr(T), len(bi), _ptr(bi), _ptr(bj), float(xi), float(dtau),
                                             float(U), f.size // N, int(n_wrap), _ptr(f), _ptr(z), int(tau), _ptr(G),
                                             ctypes.byref(la), ctypes.byref(ar)), "hubbard_ising_green_udv")
    return G[..., 0] + 1j * G[..., 1], la.value, ar.value


def bond_rank2_update(G: np.ndarray, i: int, j: int, delta: np.ndarray):
    """(G', det ratio) of the rank-2 change (1 + Delta) on the rows/columns {i, j}."""
    N = G.shape[0]
    Gi = np.ascontiguousarray(np.stack([G.real, G.imag], axis=-1), dtype=np.float64)
    d = np.asarray(delta, dtype=complex)
    dd = np.ascontiguousarray(np.stack([d.real, d.imag], axis=-1), dtype=np.float64)
    r = np.zeros(2)
    _check(lib().orc_bond_rank2_update(N, _ptr(Gi), int(i), int(j), _ptr(dd), _ptr(r)), "bond_rank2_update")
    return Gi[..., 0] + 1j * Gi[..., 1], complex(r[0], r[1])


class HubbardIsingChain:
    """A Markov chain of the Hubbard-Ising bond model (HS fields and bond spins),
    sampled with W = |Re e^{-S}| (plain recomputes; small clusters only)."""

    def __init__(self, T, bonds, xi, h, J, pairs, dtau, U, hs, ising, seed: int, chain: int):
        self.T = np.ascontiguousarray(T, dtype=np.float64)
        self.bi, self.bj = _bond_arrays(bonds)
        self.xi, self.h, self.J = float(xi), float(h), float(J)
        self.pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        self.dtau, self.U = float(dtau), float(U)
        self.hs = np.ascontiguousarray(hs, dtype=np.int8).copy()
        self.ising = np.ascontiguousarray(ising, dtype=np.int8).copy()
        self.L = self.hs.size // self.T.shape[0]
        self.seed, self.chain, self.n_sweeps = int(seed), int(chain), 0
        self.phase = np.zeros(2)

    def sweep(self):
        """One sweep; returns (reweighted Kin, sign, reweighted (sum_b s_b)^2 / n_bonds, accepted)."""
        obs = np.zeros(5)
        acc = ctypes.c_int()
        _check(lib().orc_hubbard_ising_sweep(self.T.shape[0], _ptr(self.T), len(self.bi), _ptr(self.bi),
                                             _ptr(self.bj), self.xi, self.h, self.J, len(self.pairs),
                                             _ptr(self.pairs) if len(self.pairs) else None, self.dtau, self.U, self.L,
                                             _ptr(self.hs), _ptr(self.ising), self.seed, self.chain, self.n_sweeps,
                                             _ptr(self.phase), _ptr(obs), ctypes.byref(acc)), "hubbard_ising_sweep")
        self.n_sweeps += 1
        return complex(obs[0], obs[1]), obs[2], complex(obs[3], obs[4]), acc.value


class Su2Chain:
    """A Markov chain of the SU(2) decoupling sampled with W = |Re e^{-S}| (plain
    recomputes; small clusters only)."""

    def __init__(self, K, dtau: float, U: float, fields, seed: int, chain: int):
        self.K = np.ascontiguousarray(K, dtype=np.float64)
        self.dtau, self.U = float(dtau), float(U)
        self.fields = np.ascontiguousarray(fields, dtype=np.int8).copy()
        self.L = self.fields.size // self.K.shape[0]
        self.seed, self.chain, self.n_sweeps = int(seed), int(chain), 0
        self.phase = np.zeros(2)

    def sweep(self):
        """One sweep; returns (sign * P / Re P * Ener (complex), sign, accepted)."""
        obs = np.zeros(3)
        acc = ctypes.c_int()
        _check(lib().orc_su2_sweep(self.K.shape[0], _ptr(self.K), self.dtau, self.U, self.L, _ptr(self.fields),
                                   self.seed, self.chain, self.n_sweeps, _ptr(self.phase), _ptr(obs),
                                   ctypes.byref(acc)), "su2_sweep")
        self.n_sweeps += 1
        return complex(obs[0], obs[1]), obs[2], acc.value


def szz_from_tau(obs: np.ndarray) -> np.ndarray:
    """sum_xy ph_x ph_y <S^z_x(tau) S^z_y(0)> of one configuration from the
    two-flavor (a, c, p) sums (flavor 0 = spin up, flavor 1 = spin down)."""
    m = obs[:, 0, 2] - obs[:, 1, 2]
    return (m * m[0] + obs[:, 0, 1] + obs[:, 1, 1]) / 4.0


def energy_grad(model: Model, fields: np.ndarray):
    """(Kin, Pot, Part, Ener) at G(0), dEner/dK^s (symmetric pairs) and dEner/dU."""
    f = np.ascontiguousarray(fields, dtype=np.int8)
    e = np.zeros(4)
    gK = np.zeros((model.n_flavors, model.N, model.N))
    gU = np.zeros(1)
    _check(lib().orc_energy_grad(model.cref(), _ptr(f), _ptr(e), _ptr(gK), _ptr(gU)), "energy_grad")
    return e, gK, float(gU[0])
