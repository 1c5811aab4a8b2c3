"""The multigrid preconditioner is a fixed symmetric positive definite operator (CPU).

CG needs its preconditioner B to be one fixed SPD matrix.  The library's V(1,1) cycle does,
on every level l:
- pre-smoothing z0 = omega D^-1 r;
- restriction r_c = P^T (r - G z0) to the 2 x 2-aggregated network;
- the coarse correction v = z0 + s P B_c r_c (the coarsest level solved exactly);
- post-smoothing z = v + omega D^-1 (r - G v),
with omega = 0.9 and s = 1.3 (an over-correction).

This test writes that cycle out in FP64 on dense matrices and forms B column by column
from unit vectors.  It checks that B is symmetric, that B is positive definite on the
non-floating nodes, and that B G has a much smaller condition number than the Jacobi
preconditioner's D^-1 G (below 20 against thousands).  Two and three levels are used, with
the coarsest of at most 1,024 nodes as in the library; the three-level case stops at 512 nodes
instead, so that its dense matrices stay small (where coarsening stops does not change the
cycle's algebra).
"""
import os
import sys

import numpy as np
import pytest

from oracle import network
from paper_2607_05818_gb300 import instances as I

sys.path.insert(0, os.path.dirname(__file__))
from mg_rules import aggregate  # noqa: E402

OMEGA, SCALE, COARSEST = 0.9, 1.3, 1024


def hierarchy(inst, coarsest=COARSEST):
    levels = [inst]
    while levels[-1].n > coarsest and max(levels[-1].W, levels[-1].H) > 1:
        levels.append(aggregate(levels[-1]))
    return levels


def prolongation(inst):
    T, W, H = inst.T, inst.W, inst.H
    Wc, Hc = (W + 1) // 2, (H + 1) // 2
    fl = network.floating_mask(inst)
    P = np.zeros((inst.n, T * Hc * Wc))
    for t in range(T):
        for y in range(H):
            for x in range(W):
                i = (t * H + y) * W + x
                if not fl[i]:
                    P[i, (t * Hc + y // 2) * Wc + x // 2] = 1.0
    return P


def vcycle_matrix(levels):
    """B of the V(1,1) cycle over `levels`, as a dense matrix: the cycle applied to every
    column of the identity at once (it is linear)."""
    Gs = [network.conductance_matrix(lv).tocsr() for lv in levels]
    Ps = [prolongation(lv) for lv in levels[:-1]]
    # coarsest: the exact inverse on its non-floating nodes (zero rows/columns elsewhere)
    Gc = Gs[-1].toarray()
    keep = np.flatnonzero(~network.floating_mask(levels[-1]))
    Bc = np.zeros_like(Gc)
    Bc[np.ix_(keep, keep)] = np.linalg.inv(Gc[np.ix_(keep, keep)])

    def apply(l, R):
        if l == len(levels) - 1:
            return Bc @ R
        G = Gs[l]
        d = G.diagonal()
        S = np.where(d > 0, OMEGA / np.where(d > 0, d, 1.0), 0.0)[:, None]
        z0 = S * R
        zc = apply(l + 1, Ps[l].T @ (R - G @ z0))
        v = z0 + SCALE * (Ps[l] @ zc)
        return v + S * (R - G @ v)

    return apply(0, np.eye(levels[0].n))


CASES = [
    ("2x36x30_two_levels", lambda: I.random_small(np.random.default_rng(41), T=2, W=36, H=30, n_tsv=30, n_pads=3), 2,
     COARSEST),
    ("1x48x44_three_levels", lambda: I.random_small(np.random.default_rng(42), T=1, W=48, H=44, n_pads=2,
                                                    open_frac=0.05), 3, 512),
    ("3x17x23_ragged", lambda: I.random_small(np.random.default_rng(43), T=3, W=17, H=23, n_tsv=40, n_pads=2), 2,
     COARSEST),
]


@pytest.mark.parametrize("name,make,nlev,coarsest", CASES, ids=[c[0] for c in CASES])
def test_vcycle_is_spd_and_preconditions(name, make, nlev, coarsest):
    inst = make()
    levels = hierarchy(inst, coarsest)
    assert len(levels) == nlev
    B = vcycle_matrix(levels)
    assert np.max(np.abs(B - B.T)) <= 1e-10 * np.max(np.abs(B))
    keep = np.flatnonzero(~network.floating_mask(inst))
    Bk = B[np.ix_(keep, keep)]
    G = network.conductance_matrix(inst).toarray()[np.ix_(keep, keep)]
    assert np.linalg.eigvalsh(0.5 * (Bk + Bk.T)).min() > 0
    # condition numbers of the preconditioned operators (similar to symmetric ones)
    Lb = np.linalg.cholesky(0.5 * (Bk + Bk.T))
    ev_mg = np.linalg.eigvalsh(Lb.T @ G @ Lb)
    dh = 1.0 / np.sqrt(np.diag(G))
    ev_j = np.linalg.eigvalsh(dh[:, None] * G * dh[None, :])
    kappa_mg, kappa_j = ev_mg.max() / ev_mg.min(), ev_j.max() / ev_j.min()
    # measured: 4.1, 5.3 and 3.5 against 4,656, 7,320 and 16,410 for Jacobi
    assert kappa_mg < 20 and kappa_mg * 100 < kappa_j, (kappa_mg, kappa_j)
