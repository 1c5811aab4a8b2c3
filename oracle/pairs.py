"""Pairwise effective resistance and IR drop of a grounded PDN (test infrastructure).

Paper Sec. II-B, Eq. 2 defines R(a, b) = (e_a - e_b)^T L^+ (e_a - e_b) on the network's
Laplacian.  With the ideal supply as an extra node that is grounded (its row and column
deleted), the Laplacian becomes G = B^T W B + D (Sec. II-A, Eq. 1 form) and, for any two
network nodes u, v (the supply plays no role in e_u - e_v),

    R(u, v) = (e_u - e_v)^T G^-1 (e_u - e_v) = Ginv_uu + Ginv_vv - 2 Ginv_uv,

which is Eq. 4 read backwards ((G_b^-1)_jk = (R_bj + R_bk - R_jk) / 2 with b the supply).
Paths through the supply count: two pads are joined through it.

IR drop (Sec. II-A, Eq. 1): G V = I with the supply as reference, so a current I_l drawn
at each load node l lowers node i's voltage by drop_i = (G^-1 I)_i.

From the solved sketch Z = G^-1 Y^T (Y^T = M^T Q^T, E[Q^T Q] = I), Z Z^T estimates G^-1,
so the same-seed JL estimates are
    R_JL(u, v) = ||Z_u - Z_v||^2,        drop_JL = Z (Z^T I).
Nodes without a conducting path to a pad are excluded: any pair touching one, and the
drop at one, is +inf; currents drawn at them are ignored (their Z rows are 0).

Through-bump currents (Sec. IV-B's TSV-planning statistic): a pad of conductance g at a
node whose voltage drops by drop_i carries g * drop_i from the supply into the network;
by Kirchhoff's current law the pad currents add up to the total load current.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as sla

from . import exact, network


def pair_reff_exact(inst, us, vs):
    """(len(us), len(vs)) exact R(u, v) from the dense inverse of G (small networks)."""
    Ginv, keep = exact.dense_inverse(inst)
    n = inst.T * inst.W * inst.H
    pos = np.full(n, -1, dtype=np.int64)
    pos[keep] = np.arange(len(keep))
    us, vs = np.asarray(us, np.int64), np.asarray(vs, np.int64)
    out = np.full((len(us), len(vs)), np.inf)
    for a, u in enumerate(us):
        if pos[u] < 0:
            continue
        for b, v in enumerate(vs):
            if pos[v] < 0:
                continue
            pu, pv = pos[u], pos[v]
            out[a, b] = Ginv[pu, pu] + Ginv[pv, pv] - 2.0 * Ginv[pu, pv]
    return out


def pair_reff_jl(Z, floating, us, vs):
    """(len(us), len(vs)) same-seed estimate R_JL(u, v) = sum_j (Z_uj - Z_vj)^2."""
    us, vs = np.asarray(us, np.int64), np.asarray(vs, np.int64)
    out = np.empty((len(us), len(vs)))
    for a, u in enumerate(us):
        d = Z[vs] - Z[u][None, :]
        out[a] = np.sum(d * d, axis=1)
    out[np.asarray(floating)[us], :] = np.inf
    out[:, np.asarray(floating)[vs]] = np.inf
    return out


def _currents(n, loads, I):
    """Dense (n, S) injection matrix: column s holds I[l, s] at node loads[l] (summed)."""
    I = np.asarray(I, np.float64)
    I = I[:, None] if I.ndim == 1 else I
    b = np.zeros((n, I.shape[1]))
    np.add.at(b, np.asarray(loads, np.int64), I)
    return b


def ir_drop_exact(inst, loads, I):
    """(n, S) exact drop = G^-1 I by a sparse direct solve; +inf at floating nodes."""
    n = inst.T * inst.W * inst.H
    G, keep, fl = network.reduced(inst)
    b = _currents(n, loads, I)
    out = np.full(b.shape, np.inf)
    lu = sla.splu(G.tocsc())
    out[keep] = lu.solve(np.ascontiguousarray(b[keep]))
    return out


def ir_drop_jl(Z, floating, loads, I):
    """(n, S) same-seed estimate drop_JL = Z (Z^T I); currents at floating nodes have zero
    rows of Z and so contribute nothing; +inf at floating nodes."""
    n = Z.shape[0]
    b = _currents(n, loads, I)
    w = Z.T @ b
    out = Z @ w
    out[np.asarray(floating)] = np.inf
    return out


def pad_currents(inst, drop):
    """(n_pads, S) current through every pad (input order): g_pad * drop at its node."""
    n_w = inst.W * inst.H
    node = (np.asarray(inst.pad_tier, np.int64) * inst.H + np.asarray(inst.pad_y, np.int64)) * inst.W \
        + np.asarray(inst.pad_x, np.int64)
    assert node.max(initial=-1) < inst.T * n_w
    d = np.asarray(drop, np.float64)
    d = d[:, None] if d.ndim == 1 else d
    return np.asarray(inst.pad_g, np.float64)[:, None] * d[node]


def bumps_for_share(currents, share=0.95):
    """Fraction of pads that together carry `share` of the total current, largest first
    (the statistic quoted for the band-like and uniform TSV placements)."""
    c = np.sort(np.abs(np.asarray(currents, np.float64)))[::-1]
    tot = c.sum()
    if tot <= 0:
        return 0.0
    k = int(np.searchsorted(np.cumsum(c), share * tot - 1e-12 * tot)) + 1
    return min(k, len(c)) / len(c)
