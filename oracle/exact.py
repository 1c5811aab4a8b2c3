"""Exact effective resistance of every node to the supply (test infrastructure).

Paper Sec. II-B, Eq. 2: R(a, b) = (e_a - e_b)^T L^+ (e_a - e_b).  With the supply
s as an extra Laplacian node and its row/column deleted (grounded), the same
quantity is R_i = R(i, s) = e_i^T G^-1 e_i, G = B^T W B + D (Eq. 1 form).  This
module computes diag(G^-1) by three independent routes:

  reff_dense        dense Cholesky G = L L^T (LAPACK as the factorisation step),
                    diag(G^-1)_i = ||L^-1 e_i||^2
  reff_gauss_jordan brute-force Gauss-Jordan inverse written out here (tiny n)
  reff_pinv         Eq. 2 literally: pseudo-inverse of the (n+1)-node Laplacian
and, for networks too large for dense algebra, exact values at sampled nodes by
sparse direct solves (SuperLU as the factorisation step): R_i = (G^-1 e_i)_i.

Floating nodes (no conducting path to a pad) are excluded and get R = +inf.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as la
import scipy.sparse.linalg as sla

from . import network


def reff_dense(inst):
    """Exact R_i for every node by dense Cholesky of G (n up to a few thousand)."""
    n = inst.T * inst.W * inst.H
    fl = network.floating_mask(inst)
    keep = np.flatnonzero(~fl)
    G = network.conductance_matrix(inst, dense=True)[np.ix_(keep, keep)]
    L = np.linalg.cholesky(G)
    Linv = la.solve_triangular(L, np.eye(len(keep)), lower=True)
    R = np.full(n, np.inf)
    R[keep] = np.sum(Linv * Linv, axis=0)
    return R


def dense_inverse(inst):
    """(G^-1 over kept nodes, kept index array) by Cholesky."""
    fl = network.floating_mask(inst)
    keep = np.flatnonzero(~fl)
    G = network.conductance_matrix(inst, dense=True)[np.ix_(keep, keep)]
    c = la.cho_factor(G, lower=True)
    return la.cho_solve(c, np.eye(len(keep))), keep


def gauss_jordan_inverse(A):
    """Inverse of a small SPD matrix by Gauss-Jordan elimination with partial pivoting."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    M = np.hstack([A, np.eye(n)])
    for c in range(n):
        p = c + int(np.argmax(np.abs(M[c:, c])))
        if p != c:
            M[[c, p]] = M[[p, c]]
        M[c] = M[c] / M[c, c]
        for r in range(n):
            if r != c and M[r, c] != 0.0:
                M[r] = M[r] - M[r, c] * M[c]
    return M[:, n:]


def reff_gauss_jordan(inst):
    n = inst.T * inst.W * inst.H
    fl = network.floating_mask(inst)
    keep = np.flatnonzero(~fl)
    G = network.conductance_matrix(inst, dense=True)[np.ix_(keep, keep)]
    Ginv = gauss_jordan_inverse(G)
    R = np.full(n, np.inf)
    R[keep] = np.diag(Ginv)
    return R


def laplacian_pinv(L, n_components=1):
    """Moore-Penrose pseudo-inverse of a graph Laplacian from its eigendecomposition:
    L^+ = sum over the non-null eigenpairs of v v^T / lambda.  A Laplacian with c
    connected components has exactly c zero eigenvalues (the smallest c of eigh)."""
    lam, V = np.linalg.eigh(L)
    lam, V = lam[n_components:], V[:, n_components:]
    return (V / lam) @ V.T


def reff_pinv(inst):
    """Eq. 2 with b = the supply node: R_i = (e_i - e_s)^T L^+ (e_i - e_s).

    Only for networks where every node reaches the supply (one component)."""
    n = inst.T * inst.W * inst.H
    Lp = laplacian_pinv(network.laplacian_with_supply(inst))
    i = np.arange(n)
    return Lp[i, i] + Lp[n, n] - 2.0 * Lp[i, n]


def pair_reff_pinv(L, a, b, n_components=1):
    """Eq. 2 for one pair on a given (connected) Laplacian."""
    e = np.zeros(L.shape[0])
    e[a] += 1.0
    e[b] -= 1.0
    return float(e @ laplacian_pinv(L, n_components) @ e)


class SparseFactor:
    """Sparse LU of G restricted to the non-floating nodes, for exact solves at sampled nodes."""

    def __init__(self, inst):
        self.n = inst.T * inst.W * inst.H
        self.G, self.keep, self.floating = network.reduced(inst)
        self.pos = np.full(self.n, -1, dtype=np.int64)
        self.pos[self.keep] = np.arange(len(self.keep))
        self.lu = sla.splu(self.G, permc_spec="MMD_AT_PLUS_A", options=dict(SymmetricMode=True))

    def green(self, i):
        """u = G^-1 e_i over all n nodes (0 at floating nodes)."""
        e = np.zeros(len(self.keep))
        e[self.pos[i]] = 1.0
        u = np.zeros(self.n)
        u[self.keep] = self.lu.solve(e)
        return u

    def reff(self, i):
        if self.floating[i]:
            return np.inf
        return float(self.green(i)[i])

    def solve(self, B):
        """X = G^-1 B for B of shape (n, k); rows of floating nodes are returned as 0."""
        X = np.zeros_like(B, dtype=np.float64)
        X[self.keep] = self.lu.solve(np.asarray(B, dtype=np.float64)[self.keep])
        return X
