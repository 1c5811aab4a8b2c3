"""The conductance matrix of a multi-tier PDN with its pads grounded (test infrastructure).

Paper Sec. II-A, Eq. 1: DC analysis of a resistive PDN is G V = I with G sparse
symmetric positive definite.  Here every wire segment, TSV segment and pad is an
edge e of conductance w_e; pads join a node to the ideal supply s.  With the
supply as an extra node the Laplacian is L = sum_e w_e b_e b_e^T (n+1 nodes);
deleting s's row and column (grounding the supply) gives
    G = B^T W B + D,
where B holds the mesh/TSV edges (+1 at the lower node id, -1 at the higher)
and D = diag(pad conductance per node).

Canonical edge numbering (every slot gets an id, open slots carry w = 0):
  x-segments: e = (t*H + y)*(W-1) + x                      for x < W-1
  y-segments: e = T*H*(W-1) + (t*(H-1) + y)*W + x          for y < H-1
  TSVs:       e = T*H*(W-1) + T*(H-1)*W + input index
  pads:       e = (previous) + n_tsv + input index
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def node_id(T, W, H, t, y, x):
    return (np.asarray(t, np.int64) * H + np.asarray(y, np.int64)) * W + np.asarray(x, np.int64)


def edge_list(inst):
    """All edges in canonical order.

    Returns (u, v, w, eid) for two-ended edges with u < v, and (pu, pw, peid)
    for pad edges (node to supply).  Open slots (w = 0) are kept, so eid is the
    canonical id above.
    """
    T, W, H = inst.T, inst.W, inst.H
    t, y, x = np.meshgrid(np.arange(T), np.arange(H), np.arange(W - 1), indexing="ij")
    ux = node_id(T, W, H, t, y, x).ravel()
    vx = ux + 1
    wx = np.asarray(inst.gx, np.float64).ravel()
    t, y, x = np.meshgrid(np.arange(T), np.arange(H - 1), np.arange(W), indexing="ij")
    uy = node_id(T, W, H, t, y, x).ravel()
    vy = uy + W
    wy = np.asarray(inst.gy, np.float64).ravel()
    ut = node_id(T, W, H, inst.tsv_tier, inst.tsv_y, inst.tsv_x).ravel()
    vt = ut + W * H
    wt = np.asarray(inst.tsv_g, np.float64).ravel()
    u = np.concatenate([ux, uy, ut])
    v = np.concatenate([vx, vy, vt])
    w = np.concatenate([wx, wy, wt])
    eid = np.arange(len(u), dtype=np.int64)
    pu = node_id(T, W, H, inst.pad_tier, inst.pad_y, inst.pad_x).ravel()
    pw = np.asarray(inst.pad_g, np.float64).ravel()
    peid = len(u) + np.arange(len(pu), dtype=np.int64)
    return u, v, w, eid, pu, pw, peid


def floating_mask(inst):
    """True for nodes with no conducting path to any pad (the paper is silent on this case:
    such nodes make G singular; they are excluded and get R = +inf).

    Connected components of the conducting edges with the supply as node n
    (scipy.sparse.csgraph as the library step)."""
    from scipy.sparse.csgraph import connected_components
    n = inst.T * inst.W * inst.H
    u, v, w, _, pu, pw, _ = edge_list(inst)
    a = np.concatenate([u[w > 0], pu[pw > 0]])
    b = np.concatenate([v[w > 0], np.full(int(np.sum(pw > 0)), n)])
    A = sp.coo_matrix((np.ones(len(a)), (a, b)), shape=(n + 1, n + 1))
    _, lab = connected_components(A, directed=False)
    return lab[:n] != lab[n]


def conductance_matrix(inst, dense=False):
    """G = B^T W B + D over all n nodes (floating nodes included, so G may be singular)."""
    n = inst.T * inst.W * inst.H
    u, v, w, _, pu, pw, _ = edge_list(inst)
    rows = np.concatenate([u, v, u, v, pu])
    cols = np.concatenate([u, v, v, u, pu])
    vals = np.concatenate([w, w, -w, -w, pw])
    G = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    G.sum_duplicates()
    return G.toarray() if dense else G


def laplacian_with_supply(inst):
    """Dense Laplacian on n+1 nodes; the supply is node n (Eq. 2 setting)."""
    n = inst.T * inst.W * inst.H
    u, v, w, _, pu, pw, _ = edge_list(inst)
    L = np.zeros((n + 1, n + 1))
    for a, b, g in zip(np.concatenate([u, pu]), np.concatenate([v, np.full(len(pu), n)]),
                       np.concatenate([w, pw])):
        L[a, a] += g
        L[b, b] += g
        L[a, b] -= g
        L[b, a] -= g
    return L


def reduced(inst):
    """(G restricted to non-floating nodes as CSR, index array of kept nodes, floating mask)."""
    fl = floating_mask(inst)
    keep = np.flatnonzero(~fl)
    G = conductance_matrix(inst)
    return G[keep][:, keep].tocsc(), keep, fl
