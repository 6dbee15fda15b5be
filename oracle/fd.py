"""Algorithms 1 and 3: fast diagonalization (oracle; test infrastructure).

Generalized eigendecomposition K_k U_k = M_k U_k D_k with U_k^T M_k U_k = I
through the Cholesky route of Section 4.1: M = L L^T, K~ = L^{-1} K L^{-T},
K~ = U~ D U~^T (orthonormal U~), U = L^{-T} U~.

Reading of Algorithm 3: from U^T M U = I and U^T K U = D the 3D operator
factors as P = (U1 (x) U2 (x) U3)^{-T} Lambda (U1 (x) U2 (x) U3)^{-1}, so
P^{-1} = (x)U_k Lambda^{-1} (x)U_k^T: the forward step applies U_k^T and the
backward step U_k (the printed algorithm has the transposes swapped; the 2D
Algorithm 1 has them this way round).

Eigenvalues are sorted ascending and each eigenvector column is signed so
that its entry of largest magnitude is positive (the paper fixes neither).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def generalized_eig(K, M):
    """(D, U) with K U = M U diag(D), U^T M U = I, by Cholesky + symmetric
    eigen-solve (Section 4.1)."""
    L = np.linalg.cholesky(M)
    T = sla.solve_triangular(L, K, lower=True)            # L^{-1} K
    Kt = sla.solve_triangular(L, T.T, lower=True).T        # L^{-1} K L^{-T}
    Kt = 0.5 * (Kt + Kt.T)
    D, Ut = np.linalg.eigh(Kt)
    U = sla.solve_triangular(L.T, Ut, lower=False)         # L^{-T} U~
    order = np.argsort(D, kind="stable")
    D, U = D[order], U[:, order]
    piv = np.argmax(np.abs(U), axis=0)
    U = U * np.sign(U[piv, np.arange(U.shape[1])])[None, :]
    return D, U


def mode_product(X, W, k, d):
    """Multiply the tensor X[i_d, ..., i_1] along direction k (0-based,
    direction 1 = the last array axis) by the matrix W: Y_j = sum_a W[j, a] X_a."""
    ax = d - 1 - k
    return np.moveaxis(np.tensordot(W, X, axes=([1], [ax])), 0, ax)


class FD:
    """Fast-diagonalization solver of P s = r (Algorithms 1 and 3)."""

    def __init__(self, pencils):
        self.d = len(pencils)
        self.eig = [generalized_eig(K, M) for (K, M) in pencils]
        self.n = [len(D) for D, _ in self.eig]
        lam = 0.0
        for k, (D, _) in enumerate(self.eig):
            shape = [1] * self.d
            shape[self.d - 1 - k] = len(D)
            lam = lam + D.reshape(shape)
        self.lam = lam                                   # D_1 (+) ... (+) D_d

    def apply(self, r):
        d = self.d
        R = np.asarray(r, dtype=np.float64).reshape(tuple(reversed(self.n)))
        for k in range(d):                               # r~ = (x)U_k^T r
            R = mode_product(R, self.eig[k][1].T, k, d)
        R = R / self.lam                                 # divide by D_1 (+) ... (+) D_d
        for k in range(d):                               # s = (x)U_k s~
            R = mode_product(R, self.eig[k][1], k, d)
        return R.ravel()
