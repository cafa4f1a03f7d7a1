"""Seeded synthetic inputs: lattices, model descriptions and field configurations.

This module holds none of the method's arithmetic.  It builds the hopping
matrices of the paper's example lattices and the seeded field arrays that both
the CUDA library and the FP64 oracle take as inputs:

* square lattice with periodic boundaries (the nearest-neighbour loop of the
  square-lattice Hubbard example, Sec. 6.1 ``Ham_hop``; next-nearest t' added on
  the two diagonals), chemical potential -mu on the diagonal;
* honeycomb lattice (Sec. 6.3): triangular Bravais lattice a1 = (1,0),
  a2 = (1/2, sqrt 3/2), two orbitals per cell, A(I)-B(I), A(I)-B(I+a1-a2),
  A(I)-B(I-a2) bonds, super-index (cell, orbital) -> 2*cell + orbital;
* open or periodic chains for the small exact-enumeration clusters.

Matrix elements are *set* (not accumulated) per bond, as in the paper's
``Op_T%O(I,J) = -t`` assignments, so a 2-wide periodic direction carries one
bond of amplitude -t between the two sites.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

FIELD_ISING = 1
FIELD_HS4 = 2


def square_lattice(Lx: int, Ly: int, t: float = 1.0, tp: float = 0.0, mu: float = 0.0) -> np.ndarray:
    """Hopping matrix K (N x N, N = Lx*Ly) of the periodic square lattice.

    Site index i = x + Lx*y.  K_ij = -t on nearest-neighbour bonds, -tp on the
    two diagonals (next-nearest), K_ii = -mu.
    """
    N = Lx * Ly
    K = np.zeros((N, N))

    def idx(x, y):
        return (x % Lx) + Lx * (y % Ly)

    for y in range(Ly):
        for x in range(Lx):
            i = idx(x, y)
            for (dx, dy, amp) in ((1, 0, t), (0, 1, t), (1, 1, tp), (1, -1, tp)):
                if amp == 0.0:
                    continue
                j = idx(x + dx, y + dy)
                if j == i:
                    continue
                K[i, j] = -amp
                K[j, i] = -amp
            K[i, i] = -mu
    return K


def honeycomb_lattice(L1: int, L2: int, t: float = 1.0, mu: float = 0.0) -> np.ndarray:
    """Hopping matrix of the periodic honeycomb lattice with L1 x L2 unit cells.

    Cell I = n1 + L1*n2 at R = n1 a1 + n2 a2; orbital A -> 2I, B -> 2I+1.
    """
    ncell = L1 * L2
    N = 2 * ncell
    K = np.zeros((N, N))

    def cell(n1, n2):
        return (n1 % L1) + L1 * (n2 % L2)

    for n2 in range(L2):
        for n1 in range(L1):
            I = cell(n1, n2)
            A = 2 * I
            K[A, A] = -mu
            K[A + 1, A + 1] = -mu
            for (d1, d2) in ((0, 0), (1, -1), (0, -1)):
                B = 2 * cell(n1 + d1, n2 + d2) + 1
                K[A, B] = -t
                K[B, A] = -t
    return K


def chain_lattice(N: int, t: float = 1.0, mu: float = 0.0, periodic: bool = False) -> np.ndarray:
    K = np.zeros((N, N))
    for i in range(N - 1):
        K[i, i + 1] = K[i + 1, i] = -t
    if periodic and N > 2:
        K[0, N - 1] = K[N - 1, 0] = -t
    np.fill_diagonal(K, -mu)
    return K


def sublattice_signs_square(Lx: int, Ly: int) -> np.ndarray:
    return np.array([(-1.0) ** (x + y) for y in range(Ly) for x in range(Lx)])


def sublattice_signs_honeycomb(L1: int, L2: int) -> np.ndarray:
    return np.array([1.0 if (i % 2 == 0) else -1.0 for i in range(2 * L1 * L2)])


def translation_classes_square(Lx: int, Ly: int):
    """Pair classes of the periodic square lattice by displacement: the pair
    (i, j) belongs to class (dx mod Lx) + Lx (dy mod Ly), dx = x_j - x_i.
    Returns (class map [N*N] int32, number of classes N, displacement r[N, 2])."""
    N = Lx * Ly
    cls = np.zeros((N, N), dtype=np.int32)
    for i in range(N):
        xi, yi = i % Lx, i // Lx
        for j in range(N):
            xj, yj = j % Lx, j // Lx
            cls[i, j] = ((xj - xi) % Lx) + Lx * ((yj - yi) % Ly)
    r = np.array([[c % Lx, c // Lx] for c in range(N)], dtype=np.float64)
    return cls.ravel(), N, r


def translation_classes_honeycomb(L1: int, L2: int):
    """Pair classes of the periodic honeycomb lattice by cell displacement and
    orbital pair: class = 4 ((d1 mod L1) + L1 (d2 mod L2)) + 2 o_i + o_j.
    Returns (class map [N*N], number of classes 4 L1 L2, displacement r[n, 2] in
    units of a1, a2 (cell part only))."""
    ncell = L1 * L2
    N = 2 * ncell
    cls = np.zeros((N, N), dtype=np.int32)
    for i in range(N):
        ci, oi = divmod(i, 2)
        n1i, n2i = ci % L1, ci // L1
        for j in range(N):
            cj, oj = divmod(j, 2)
            n1j, n2j = cj % L1, cj // L1
            d = ((n1j - n1i) % L1) + L1 * ((n2j - n2i) % L2)
            cls[i, j] = 4 * d + 2 * oi + oj
    r = np.array([[(c // 4) % L1, (c // 4) // L1] for c in range(4 * ncell)], dtype=np.float64)
    return cls.ravel(), 4 * ncell, r


@dataclass
class ModelSpec:
    """One Hubbard model in the spin-z decoupling: flavors up (+1) and down (-1)."""

    hopping: np.ndarray                 # [N, N] shared by both flavors (or [2, N, N])
    U: float
    dtau: float
    L: int
    n_wrap: int = 10
    field_type: int = FIELD_ISING
    name: str = ""
    vertex_site: np.ndarray | None = None
    vertex_sign: np.ndarray | None = None

    def __post_init__(self):
        H = np.asarray(self.hopping, dtype=np.float64)
        if H.ndim == 2:
            H = np.stack([H, H])
        self.hopping = np.ascontiguousarray(H)
        N = H.shape[-1]
        if self.vertex_site is None:
            self.vertex_site = np.arange(N, dtype=np.int32)
        if self.vertex_sign is None:
            MV = len(self.vertex_site)
            self.vertex_sign = np.stack([np.ones(MV), -np.ones(MV)])[: H.shape[0]]
        self.vertex_site = np.ascontiguousarray(self.vertex_site, dtype=np.int32)
        self.vertex_sign = np.ascontiguousarray(self.vertex_sign, dtype=np.float64)

    @property
    def N(self) -> int:
        return int(self.hopping.shape[-1])

    @property
    def n_vertices(self) -> int:
        return int(len(self.vertex_site))

    @property
    def beta(self) -> float:
        return self.L * self.dtau


def random_fields(field_type: int, L: int, MV: int, seed: int) -> np.ndarray:
    """Seeded i.i.d. uniform fields [L, MV] (numpy PCG64): +-1, or -2,-1,1,2."""
    rng = np.random.default_rng(seed)
    if field_type == FIELD_ISING:
        return (2 * rng.integers(0, 2, size=(L, MV)) - 1).astype(np.int8)
    vals = np.array([-2, -1, 1, 2], dtype=np.int8)
    return vals[rng.integers(0, 4, size=(L, MV))]


BASE_SEED = 20170401


@dataclass
class Workload:
    """A set of chains, each referring to one model."""

    name: str
    models: list = field(default_factory=list)
    chain_model: np.ndarray | None = None
    precision: str = "fp64"            # "fp64" or "mixed"
    delay_k: int = 16

    @property
    def n_chains(self) -> int:
        return int(len(self.chain_model))

    def proposals_per_sweep(self) -> int:
        return int(sum(2 * self.models[m].L * self.models[m].n_vertices for m in self.chain_model))


def config_c1() -> Workload:
    """4x4 square Hubbard, t=1, U=4, mu=0, beta=2, dtau=0.1 (L=20), Ising HS, n_wrap=10, 1 chain."""
    m = ModelSpec(square_lattice(4, 4), U=4.0, dtau=0.1, L=20, n_wrap=10, name="square4x4_U4_b2")
    return Workload("square 4x4 L=20 (1 chain, FP64)", [m], np.zeros(1, dtype=np.int32), "fp64", 1)


def config_c2() -> Workload:
    """Honeycomb 6x6 cells (N=72), t=1, U=4, mu=0, beta=10, dtau=0.1 (L=100), n_wrap=10, 1 chain."""
    m = ModelSpec(honeycomb_lattice(6, 6), U=4.0, dtau=0.1, L=100, n_wrap=10, name="honeycomb6x6_U4_b10")
    return Workload("honeycomb 6x6 L=100 (1 chain, FP64)", [m], np.zeros(1, dtype=np.int32), "fp64", 1)


def config_c3(n_chains: int = 256, precision: str = "mixed") -> Workload:
    """256 chains: N=64 (8x8) for c < n/2 else N=144 (12x12); beta = 4 (c even) or 8 (c odd);
    U = (2,4,6)[c mod 3]; dtau = 0.1, n_wrap = 10."""
    models = []
    key = {}
    cm = np.zeros(n_chains, dtype=np.int32)
    for c in range(n_chains):
        Ls = 8 if c < n_chains // 2 else 12
        beta = 4.0 if c % 2 == 0 else 8.0
        U = (2.0, 4.0, 6.0)[c % 3]
        k = (Ls, beta, U)
        if k not in key:
            key[k] = len(models)
            models.append(ModelSpec(square_lattice(Ls, Ls), U=U, dtau=0.1, L=int(round(beta / 0.1)), n_wrap=10,
                                    name=f"square{Ls}x{Ls}_U{U:g}_b{beta:g}"))
        cm[c] = key[k]
    return Workload(f"square 8x8/12x12 x{n_chains} chains", models, cm, precision, 16)


def config_c4() -> Workload:
    """8x8 square, beta=4, dtau=0.1 (L=40), U=4: 64 fixed seeded configurations (no MC)."""
    m = ModelSpec(square_lattice(8, 8), U=4.0, dtau=0.1, L=40, n_wrap=10, name="square8x8_U4_b4")
    return Workload("square 8x8 L=40 gradients", [m], np.zeros(64, dtype=np.int32), "fp64", 1)


def config_c5(n_chains: int = 32, precision: str = "mixed") -> Workload:
    """20x20 square (N=400), t=1, t'=-0.2, U=4, mu=-0.5, beta=10, dtau=0.05 (L=200), 32 chains, delay 32."""
    m = ModelSpec(square_lattice(20, 20, t=1.0, tp=-0.2, mu=-0.5), U=4.0, dtau=0.05, L=200, n_wrap=10,
                  name="square20x20_tp-0.2_mu-0.5_U4_b10")
    return Workload("square 20x20 L=200 x32 chains", [m], np.zeros(n_chains, dtype=np.int32), precision, 32)
