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
        g = np.sqrt(0.5 * dtau * U)
        W = np.eye(self.dim)
        for i in range(self.N):
            A = np.diag(self.n(0, i)) - np.diag(self.n(1, i))
            w = sum(gamma[l] * np.exp(g * eta[l] * A) for l in (-2, -1, 1, 2)) / 4.0
            W = W @ np.diag(w)
        return np.linalg.matrix_power(E @ W, L)
