"""The paper's own bump-to-load effective resistance through a reduced TSV system
(test infrastructure; an exact cross-check of the Cholesky route on uniform stacks).

Setting (Sec. III-C, Table "Notations"): d stacked dies, each a uniform M x N mesh
(die i: x-segments r_i, y-segments s_i); p TSVs, each a through-stack column at
(tx_k, ty_k) with segment resistance Rt_k^{i,i+1} between die i and die i+1.  A
unit current enters at the bump s^1 on die 1 and leaves at the load s^d on die d;
the reference node s^i of an intermediate die is arbitrary (its net current is 0).

Steps, in the paper's order:
  Eq. 7   intra-die voltages through a^i_{s,j,k} = (R^i_{s,j} + R^i_{s,k} - R^i_{j,k}) / 2,
          with the intra-die two-point resistances R^i from Wu's closed form (Eq. 3);
  Eq. 8-9 Ohm's law on every TSV segment plus the unit-current constraints;
  Eq. 10  the KKT system [A + D, B; B^T, 0][I; V] = [0; 1], V_i = -(V_s^i - V_s^{i+1});
  Eq. 6   R = sum_i (V_s^i - V_s^{i+1}) = -sum_i V_i.
And the pair-independent form:
  Eq. 13  [A~ + D, B; B^T, 0] x = b with A~^i = -R^i_{jk} / 2 (zero diagonal),
          b = [-R^1_{s,.}/2, 0, ..., -R^d_{s,.}/2, 1_{d-1}], R = -x^T b;
  Eq. 14-15  b = b^1 + b^d, one factorisation, m + n solves,
          R(i, j) = -(x^1_i + x^d_j)^T (b^1_i + b^d_j).

Readings (the typeset equations are garbled in places): Eq. 8 uses a exactly as
defined beside it (no extra 1/2); the off-diagonal blocks of A~ are -A~^{i+1};
b's last block is 1_{d-1} (printed as 1_p); the sums in v~_i run over the p TSVs
(printed j = 1..d-1) and carry the 1/2 of a.  With those readings R = -x^T b
follows from Eq. 6 by telescoping the v~_i.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as la

from .wu import reff_wu


class UniformStack:
    def __init__(self, M, N, r, s, tsv_xy, Rt):
        """r, s: per-die segment resistances (length d); tsv_xy: p positions;
        Rt: (d-1, p) TSV segment resistances."""
        self.M, self.N = M, N
        self.r = list(r)
        self.s = list(s)
        self.d = len(self.r)
        self.tsv = [tuple(t) for t in tsv_xy]
        self.p = len(self.tsv)
        self.Rt = np.asarray(Rt, dtype=np.float64).reshape(self.d - 1, self.p)

    def R(self, i, a, b):
        """Intra-die two-point resistance on die i (0-based) by Eq. 3."""
        return reff_wu(self.M, self.N, self.r[i], self.s[i], a, b)

    def tsv_tsv(self, i):
        P = self.p
        out = np.zeros((P, P))
        for j in range(P):
            for k in range(j + 1, P):
                out[j, k] = out[k, j] = self.R(i, self.tsv[j], self.tsv[k])
        return out

    def point_tsv(self, i, pt):
        return np.array([self.R(i, pt, t) for t in self.tsv])


def _kkt(blocks_diag, blocks_off, Rt, d, p):
    """[[X + D, B], [B^T, 0]] with X block tridiagonal: diag blocks_diag[i], off blocks_off[i]
    between block rows i and i+1."""
    nI = p * (d - 1)
    C = np.zeros((nI + d - 1, nI + d - 1))
    for i in range(d - 1):
        sl = slice(i * p, (i + 1) * p)
        C[sl, sl] = blocks_diag[i]
        if i + 1 < d - 1:
            sl2 = slice((i + 1) * p, (i + 2) * p)
            C[sl, sl2] = blocks_off[i]
            C[sl2, sl] = blocks_off[i].T
        C[sl, sl] += np.diag(Rt[i])
        C[sl, nI + i] = 1.0
        C[nI + i, sl] = 1.0
    return C


def pair_reff_kkt(st: UniformStack, bump, load, mid_ref=None):
    """Eq. 10 for one bump (die 1) / load (die d) pair; returns (R, I, V)."""
    d, p = st.d, st.p
    ref = [None] * d
    for i in range(d):
        ref[i] = bump if i == 0 else load if i == d - 1 else (mid_ref or st.tsv[0])
    A = []
    for i in range(d):
        Rss = st.point_tsv(i, ref[i])
        Rjk = st.tsv_tsv(i)
        A.append(0.5 * (Rss[:, None] + Rss[None, :] - Rjk))
    diag = [A[i] + A[i + 1] for i in range(d - 1)]
    off = [-A[i + 1] for i in range(d - 2)]
    C = _kkt(diag, off, st.Rt, d, p)
    rhs = np.zeros(C.shape[0])
    rhs[p * (d - 1):] = 1.0
    x = np.linalg.solve(C, rhs)
    I, V = x[: p * (d - 1)], x[p * (d - 1):]
    return float(-np.sum(V)), I, V


class TransformedSystem:
    """Eq. 13-15: one factorisation of the pair-independent C, then m + n solves."""

    def __init__(self, st: UniformStack):
        self.st = st
        d, p = st.d, st.p
        At = [-0.5 * st.tsv_tsv(i) for i in range(d)]
        diag = [At[i] + At[i + 1] for i in range(d - 1)]
        off = [-At[i + 1] for i in range(d - 2)]
        self.C = _kkt(diag, off, st.Rt, d, p)
        self.lu = la.lu_factor(self.C)

    def b_bump(self, bump):
        st, d, p = self.st, self.st.d, self.st.p
        b = np.zeros(self.C.shape[0])
        b[:p] = -0.5 * st.point_tsv(0, bump)
        b[p * (d - 1):] = 0.5
        return b

    def b_load(self, load):
        st, d, p = self.st, self.st.d, self.st.p
        b = np.zeros(self.C.shape[0])
        b[(d - 2) * p:(d - 1) * p] = -0.5 * st.point_tsv(d - 1, load)
        b[p * (d - 1):] = 0.5
        return b

    def pairs(self, bumps, loads):
        """m x n matrix of bump-load effective resistances (Eq. 15)."""
        B1 = np.stack([self.b_bump(b) for b in bumps], axis=1)
        Bd = np.stack([self.b_load(l) for l in loads], axis=1)
        X1 = la.lu_solve(self.lu, B1)
        Xd = la.lu_solve(self.lu, Bd)
        out = np.zeros((len(bumps), len(loads)))
        for i in range(len(bumps)):
            for j in range(len(loads)):
                out[i, j] = -(X1[:, i] + Xd[:, j]) @ (B1[:, i] + Bd[:, j])
        return out
