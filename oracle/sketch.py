"""The seeded JL sketch and the same-seed JL estimate of the R map (test infrastructure).

All-node map: R_i = e_i^T G^-1 e_i = ||M G^-1 e_i||^2 with M = [W^{1/2} B; D^{1/2}],
because M^T M = B^T W B + D = G.  A k x m Rademacher matrix Q (entries +-1/sqrt(k),
E[Q^T Q] = I) gives the estimate R_JL,i = ||Q M G^-1 e_i||^2 = ||Z_i||^2 with
Z = G^-1 Y^T, Y^T = M^T Q^T (Spielman-Srivastava sparsification sketch).  The
paper has no sketch; it defines only R itself (Sec. II-B, Eq. 2).

Q[j][e]: sign from the top bit of SplitMix64(key XOR (e * 2^32 + j)) with
key = SplitMix64(seed) (SplitMix64: Steele, Lea and Flood 2014), top bit 0 -> +1.
Mixing the seed first keeps nearby seeds from reusing each other's counters.
e is the canonical edge id of oracle.network; M's row e has +sqrt(w_e) at the lower node id and -sqrt(w_e) at
the higher one (a pad row: +sqrt(g) at its node).  Rows of floating nodes are 0.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import network

_M1 = np.uint64(0x9E3779B97F4A7C15)
_M2 = np.uint64(0xBF58476D1CE4E5B9)
_M3 = np.uint64(0x94D049BB133111EB)


def splitmix64(z):
    """SplitMix64 output function on a uint64 array (wrap-around arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z + _M1
        z = (z ^ (z >> np.uint64(30))) * _M2
        z = (z ^ (z >> np.uint64(27))) * _M3
    return z ^ (z >> np.uint64(31))


def rademacher(seed, eids, k):
    """(len(eids), k) array of +-1: sign of Q[j][e] * sqrt(k)."""
    e = np.asarray(eids, dtype=np.uint64)[:, None]
    j = np.arange(k, dtype=np.uint64)[None, :]
    key = splitmix64(np.array([seed], dtype=np.uint64))[0]
    h = splitmix64(key ^ ((e << np.uint64(32)) | j))
    return 1.0 - 2.0 * (h >> np.uint64(63)).astype(np.float64)


def sketch_numpy(inst, k, seed):
    """Y^T (n x k, FP64) by an explicit loop over edge chunks."""
    n = inst.T * inst.W * inst.H
    u, v, w, eid, pu, pw, peid = network.edge_list(inst)
    Yt = np.zeros((n, k))
    rk = 1.0 / np.sqrt(k)
    on = w > 0
    for lo in range(0, int(on.sum()), 4096):
        sel = np.flatnonzero(on)[lo:lo + 4096]
        q = rademacher(seed, eid[sel], k) * (np.sqrt(w[sel]) * rk)[:, None]
        np.add.at(Yt, u[sel], q)
        np.add.at(Yt, v[sel], -q)
    pon = np.flatnonzero(pw > 0)
    if len(pon):
        q = rademacher(seed, peid[pon], k) * (np.sqrt(pw[pon]) * rk)[:, None]
        np.add.at(Yt, pu[pon], q)
    Yt[network.floating_mask(inst)] = 0.0
    return Yt


def sketch_rows(inst, nodes, k, seed):
    """Rows `nodes` (distinct) of Y^T, (len(nodes), k) FP64: each row is the sum over its
    node's conducting edges of +-sqrt(w_e) Q[:, e] (pad edges +), so a few rows of a
    network too large for sketch_numpy cost one pass over the edge list."""
    nodes = np.asarray(nodes, dtype=np.int64)
    if len(np.unique(nodes)) != len(nodes):
        raise ValueError("nodes must be distinct")
    order = np.argsort(nodes)
    srt = nodes[order]
    u, v, w, eid, pu, pw, peid = network.edge_list(inst)
    out = np.zeros((len(nodes), k))
    rk = 1.0 / np.sqrt(k)
    for ends, sign in ((u, 1.0), (v, -1.0)):
        sel = np.flatnonzero(np.isin(ends, srt) & (w > 0))
        q = rademacher(seed, eid[sel], k) * (sign * np.sqrt(w[sel]) * rk)[:, None]
        np.add.at(out, order[np.searchsorted(srt, ends[sel])], q)
    sel = np.flatnonzero(np.isin(pu, srt) & (pw > 0))
    q = rademacher(seed, peid[sel], k) * (np.sqrt(pw[sel]) * rk)[:, None]
    np.add.at(out, order[np.searchsorted(srt, pu[sel])], q)
    out[network.floating_mask(inst)[nodes]] = 0.0
    return out


_LIB = None


def _clib():
    global _LIB
    if _LIB is None:
        path = os.path.join(os.path.dirname(__file__), "_oracle_sketch.so")
        if not os.path.exists(path):
            return None
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        lib.oracle_sketch.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.c_int64, P, P, P, P, ctypes.c_int64, P, P, P, P]
        lib.oracle_sketch.restype = None
        _LIB = lib
    return _LIB


def sketch_c(inst, k, seed):
    """Same as sketch_numpy through the plain C edge loop in csrc/oracle_sketch.c."""
    lib = _clib()
    if lib is None:
        raise RuntimeError("oracle/_oracle_sketch.so is not built (run __graft_entry__.build())")
    n = inst.T * inst.W * inst.H
    u, v, w, eid, pu, pw, peid = network.edge_list(inst)
    arr = [np.ascontiguousarray(a) for a in (u, v, w, eid, pu, pw, peid)]
    Yt = np.zeros((n, k))
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    lib.oracle_sketch(n, k, ctypes.c_uint64(int(seed)), len(arr[0]), p(arr[0]), p(arr[1]),
                      p(arr[2]), p(arr[3]), len(arr[4]), p(arr[4]), p(arr[5]), p(arr[6]), p(Yt))
    Yt[network.floating_mask(inst)] = 0.0
    return Yt


def sketch(inst, k, seed):
    """Y^T in FP64; the C loop when built, the numpy loop otherwise (they are pinned equal)."""
    if _clib() is not None:
        return sketch_c(inst, k, seed)
    return sketch_numpy(inst, k, seed)


def reff_jl_dense(inst, k, seed, Yt=None):
    """Same-seed R_JL for every node by dense Cholesky solves: Z = G^-1 Y^T, R = sum_j Z_ij^2."""
    import scipy.linalg as la
    n = inst.T * inst.W * inst.H
    Yt = sketch(inst, k, seed) if Yt is None else Yt
    fl = network.floating_mask(inst)
    keep = np.flatnonzero(~fl)
    G = network.conductance_matrix(inst, dense=True)[np.ix_(keep, keep)]
    Z = np.zeros((n, k))
    Z[keep] = la.cho_solve(la.cho_factor(G, lower=True), Yt[keep])
    R = np.full(n, np.inf)
    R[keep] = np.sum(Z[keep] * Z[keep], axis=1)
    return R, Z


def reff_jl_sampled(factor, Yt, nodes):
    """Same-seed R_JL and Z rows at sampled nodes, one exact solve each:
    Z_i = (G^-1 e_i)^T Y^T since G is symmetric."""
    R, Zs = [], []
    for i in nodes:
        if factor.floating[i]:
            R.append(np.inf)
            Zs.append(np.zeros(Yt.shape[1]))
            continue
        g = factor.green(int(i))
        z = g @ Yt
        Zs.append(z)
        R.append(float(z @ z))
    return np.array(R), np.array(Zs)
