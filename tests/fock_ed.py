"""Exact diagonalisation in the fermionic Fock space of small clusters (test helper).

Modes m = s*N + x (flavor s in {0: up, 1: down}, site x); Jordan-Wigner strings
give the anticommuting annihilation operators as dense 4^N x 4^N matrices.  It
is used to pin the oracle's determinant weights and Green functions: for a
fixed field history Tr_F[prod_tau exp(c^+ X_tau c)] = det(1 + prod_tau exp(X_tau)),
so summing the oracle's weights over all field configurations must equal the
Fock-space trace of the Trotterised density matrix.
"""
import numpy as np
from scipy.linalg import expm


def annihilators(n_modes: int):
    sz = np.diag([1.0, -1.0])
    lower = np.array([[0.0, 1.0], [0.0, 0.0]])  # |0><1| in the (|0>, |1>) basis
    eye = np.eye(2)
    ops = []
    for m in range(n_modes):
        mats = [sz] * m + [lower] + [eye] * (n_modes - m - 1)
        op = mats[0]
        for a in mats[1:]:
            op = np.kron(op, a)
        ops.append(op)
    return ops


class Fock:
    def __init__(self, N: int, n_flavors: int = 2):
        self.N = N
        self.nfl = n_flavors
        self.c = annihilators(N * n_flavors)
        self.dim = self.c[0].shape[0]

    def mode(self, s, x):
        return s * self.N + x

    def n(self, s, x):
        c = self.c[self.mode(s, x)]
        return c.T @ c

    def one_body(self, X, s):
        """c^+_s X c_s for flavor s."""
        H = np.zeros((self.dim, self.dim))
        for x in range(self.N):
            for y in range(self.N):
                if X[x, y] != 0.0:
                    H += X[x, y] * (self.c[self.mode(s, x)].T @ self.c[self.mode(s, y)])
        return H

    def hopping(self, K):
        return sum(self.one_body(K[s] if K.ndim == 3 else K, s) for s in range(self.nfl))

    def hubbard_ph(self, U):
        """U sum_i (n_up - 1/2)(n_dn - 1/2)."""
        I = np.eye(self.dim)
        return sum(U * (self.n(0, i) - 0.5 * I) @ (self.n(1, i) - 0.5 * I) for i in range(self.N))

    def hubbard_nn(self, U):
        """U sum_i n_up n_dn."""
        return sum(U * self.n(0, i) @ self.n(1, i) for i in range(self.N))

    def trotter_ising(self, K, U, dtau, L):
        """(exp(-dtau H_T) exp(-dtau H_U))^L, H_U = U sum (n_up-1/2)(n_dn-1/2)."""
        E = expm(-dtau * self.hopping(K))
        W = expm(-dtau * self.hubbard_ph(U))
        return np.linalg.matrix_power(E @ W, L)

    def trotter_hs4(self, K, U, dtau, L, eta, gamma):
        """(exp(-dtau H_T) W)^L with W = prod_i (1/4) sum_l gamma(l) exp(g eta(l) (n_up - n_dn))."""
        E = expm(-dtau * self.hopping(K))
        return np.linalg.matrix_power(E @ hs4_slice(self, U, dtau, eta, gamma), L)


def hs4_slice(F, U, dtau, eta, gamma):
    """prod_i (1/4) sum_l gamma(l) exp(g eta(l) (n_i,up - n_i,dn)), g = sqrt(dtau U / 2):
    the interaction factor of one slice after summing the four-valued field."""
    g = np.sqrt(0.5 * dtau * U)
    W = np.eye(F.dim)
    for i in range(F.N):
        A = np.diag(F.n(0, i)) - np.diag(F.n(1, i))
        W = W @ np.diag(sum(gamma[l] * np.exp(g * eta[l] * A) for l in (-2, -1, 1, 2)) / 4.0)
    return W


def tau_observables(F, K, U, dtau, L, ph, W=None):
    """Local Green function sum_s,x <c_xs(tau) c^+_xs(0)> and the phase-weighted
    sum_xy ph_x ph_y <S^z_x(tau) S^z_y(0)> for tau = 0..L of the Trotterised
    Hubbard model: <A(tau) B(0)> = Tr[T^{L-tau} A T^tau B] / Tr[T^L] with
    T = exp(-dtau H_T) W, W = exp(-dtau H_U) (exact Ising decoupling) unless given."""
    N = K.shape[0]
    if W is None:
        W = expm(-dtau * F.hubbard_ph(U))
    T = expm(-dtau * F.hopping(K)) @ W
    Z = np.trace(np.linalg.matrix_power(T, L))
    Sz = [0.5 * (F.n(0, x) - F.n(1, x)) for x in range(N)]
    SzP = sum(ph[x] * Sz[x] for x in range(N))
    gl, szz = [], []
    for tau in range(L + 1):
        A = np.linalg.matrix_power(T, L - tau)
        B = np.linalg.matrix_power(T, tau)
        g = 0.0
        for s in range(2):
            for x in range(N):
                c = F.c[F.mode(s, x)]
                g += np.trace(A @ c @ B @ c.T)
        gl.append(g / Z)
        szz.append(np.trace(A @ SzP @ B @ SzP) / Z)
    return np.array(gl), np.array(szz)


def tau_correlations(F, K, U, dtau, L, cls, n_class):
    """Per tau = 0..L and pair class: sums of sum_s <c_xs(tau) c^+_ys(0)>,
    <S^z_x(tau) S^z_y(0)> and <n_x(tau) n_y(0)> of the Trotterised Hubbard model
    (exact Ising decoupling), <A(tau) B(0)> = Tr[T^{L-tau} A T^tau B] / Tr[T^L]."""
    N = K.shape[0]
    T = expm(-dtau * F.hopping(K)) @ expm(-dtau * F.hubbard_ph(U))
    Z = np.trace(np.linalg.matrix_power(T, L))
    out = np.zeros((L + 1, n_class, 3))
    sz = [0.5 * (F.n(0, x) - F.n(1, x)) for x in range(N)]
    nn = [F.n(0, x) + F.n(1, x) for x in range(N)]
    for tau in range(L + 1):
        A = np.linalg.matrix_power(T, L - tau)
        B = np.linalg.matrix_power(T, tau)
        for x in range(N):
            for y in range(N):
                c = cls[x * N + y]
                if c < 0:
                    continue
                g = sum(np.trace(A @ F.c[F.mode(s, x)] @ B @ F.c[F.mode(s, y)].T) for s in range(2))
                out[tau, c, 0] += g / Z
                out[tau, c, 1] += np.trace(A @ sz[x] @ B @ sz[y]) / Z
                out[tau, c, 2] += np.trace(A @ nn[x] @ B @ nn[y]) / Z
    return out


def equal_time_correlations(F, K, U, dtau, L, cls, n_class):
    """Per pair class: sums of <S^z_x S^z_y>, <n_x n_y>, <S^+_x S^-_y> and
    sum_s <c^+_xs c_ys> in the Trotterised density matrix (trace boundary)."""
    N = K.shape[0]
    rho = F.trotter_ising(K, U, dtau, L)
    Z = np.trace(rho)
    out = np.zeros((n_class, 4))
    cu = [F.c[F.mode(0, x)] for x in range(N)]
    cd = [F.c[F.mode(1, x)] for x in range(N)]
    for x in range(N):
        for y in range(N):
            c = cls[x * N + y]
            szx = 0.5 * (F.n(0, x) - F.n(1, x))
            szy = 0.5 * (F.n(0, y) - F.n(1, y))
            nx = F.n(0, x) + F.n(1, x)
            ny = F.n(0, y) + F.n(1, y)
            spm = cu[x].T @ cd[x] @ cd[y].T @ cu[y]
            hop = cu[x].T @ cu[y] + cd[x].T @ cd[y]
            for q, O in enumerate((szx @ szy, nx @ ny, spm, hop)):
                out[c, q] += np.trace(O @ rho) / Z
    return out


def su2_trotter(F, K, U, dtau, L, eta, gamma):
    """Partition function and <H_T + U/2 sum_i (n_i - 1)^2> of the Trotter product
    (exp(-dtau H_T) W)^L with the summed slice factor of the SU(2) charge
    decoupling, W = prod_i sum_l gamma(l)/4 exp(i g eta(l) (n_i - 1)), g = sqrt(dtau U/2)."""
    N = K.shape[0]
    g = np.sqrt(0.5 * dtau * U)
    Wd = np.ones(F.dim, dtype=complex)
    for i in range(N):
        ni = np.diag(F.n(0, i)) + np.diag(F.n(1, i))
        Wd *= sum(gamma[l] / 4.0 * np.exp(1j * g * eta[l] * (ni - 1.0)) for l in (-2, -1, 1, 2))
    rho = np.linalg.matrix_power(expm(-dtau * F.hopping(K)) @ np.diag(Wd), L)
    I = np.eye(F.dim)
    HU = sum(0.5 * U * (F.n(0, i) + F.n(1, i) - I) @ (F.n(0, i) + F.n(1, i) - I) for i in range(N))
    Z = np.trace(rho)
    return Z, np.trace((F.hopping(K) + HU) @ rho) / Z


def hubbard_ising_trotter(F, K, U, dtau, L, eta, gamma, bonds, xi, h, J, pairs, with_m2=False):
    """Partition function and <H_T> of the Trotter product of the Hubbard model
    coupled to Ising spins on bonds, on the product space Fock (x) Ising
    (Ising basis state k: s_b = 1 - 2 bit_b(k)):
      S = exp(-dtau H_T) prod_b exp(-dtau xi Z_b O_b) W exp(dtau J sum_pairs Z Z) prod_b exp(dtau h X_b),
    O_b = sum_s (c^+_is c_js + h.c.), W the summed slice factor of the SU(2)
    charge decoupling.  Returns (Tr S^L, Tr[H_T S^L] / Tr S^L) and, with
    with_m2, <(sum_b Z_b)^2> / n_bonds as a third value."""
    N = K.shape[0]
    nb = len(bonds)
    dI = 2 ** nb
    s = np.array([[1.0 - 2.0 * ((k >> b) & 1) for b in range(nb)] for k in range(dI)])   # [dI, nb]
    If = np.eye(F.dim)
    g = np.sqrt(0.5 * dtau * U)
    Wd = np.ones(F.dim, dtype=complex)
    for i in range(N):
        ni = np.diag(F.n(0, i)) + np.diag(F.n(1, i))
        Wd *= sum(gamma[l] / 4.0 * np.exp(1j * g * eta[l] * (ni - 1.0)) for l in (-2, -1, 1, 2))
    S = np.kron(expm(-dtau * F.hopping(K)), np.eye(dI)).astype(complex)
    for b, (i, j) in enumerate(bonds):
        Ob = np.zeros((N, N))
        Ob[i, j] = Ob[j, i] = 1.0
        S = S @ expm(-dtau * xi * np.kron(F.hopping(Ob), np.diag(s[:, b])))
    S = S @ np.kron(np.diag(Wd), np.eye(dI))
    zz = np.array([sum(s[k, p] * s[k, q] for p, q in pairs) for k in range(dI)])
    S = S @ np.kron(If, np.diag(np.exp(dtau * J * zz)))
    for b in range(nb):
        Xb = np.zeros((dI, dI))
        for k in range(dI):
            Xb[k ^ (1 << b), k] = 1.0
        S = S @ np.kron(If, expm(dtau * h * Xb))
    rho = np.linalg.matrix_power(S, L)
    Z = np.trace(rho)
    kin = np.trace(np.kron(F.hopping(K), np.eye(dI)) @ rho) / Z
    if not with_m2:
        return Z, kin
    m2 = np.kron(np.ones(F.dim), s.sum(axis=1) ** 2 / nb)
    return Z, kin, np.trace(np.diag(m2) @ rho) / Z


def su2_correlations(F, K, U, dtau, L, eta, gamma, cls, n_class):
    """Per pair class: sums of <S^z_x S^z_y>, <n_x n_y>, <S^+_x S^-_y> and
    sum_s <c^+_xs c_ys> in the Trotter product of the SU(2) charge decoupling
    (summed slice factor W as su2_trotter), at the trace boundary."""
    N = K.shape[0]
    g = np.sqrt(0.5 * dtau * U)
    Wd = np.ones(F.dim, dtype=complex)
    for i in range(N):
        ni = np.diag(F.n(0, i)) + np.diag(F.n(1, i))
        Wd *= sum(gamma[l] / 4.0 * np.exp(1j * g * eta[l] * (ni - 1.0)) for l in (-2, -1, 1, 2))
    rho = np.linalg.matrix_power(expm(-dtau * F.hopping(K)) @ np.diag(Wd), L)
    Z = np.trace(rho)
    out = np.zeros((n_class, 4), dtype=complex)
    cu = [F.c[F.mode(0, x)] for x in range(N)]
    cd = [F.c[F.mode(1, x)] for x in range(N)]
    for x in range(N):
        for y in range(N):
            c = cls[x * N + y]
            szx = 0.5 * (F.n(0, x) - F.n(1, x))
            szy = 0.5 * (F.n(0, y) - F.n(1, y))
            nx = F.n(0, x) + F.n(1, x)
            ny = F.n(0, y) + F.n(1, y)
            spm = cu[x].T @ cd[x] @ cd[y].T @ cu[y]
            hop = cu[x].T @ cu[y] + cd[x].T @ cd[y]
            for q, O in enumerate((szx @ szy, nx @ ny, spm, hop)):
                out[c, q] += np.trace(O @ rho) / Z
    return out
