"""The multigrid's aggregation rule, written out for the CPU tests (a helper module, not a
test): the coarse network of 2 x 2 aggregation and the Galerkin product P^T G P."""
import numpy as np

from oracle import network
from paper_2607_05818_gb300 import instances as I


def aggregate(inst):
    """The coarse instance by the aggregation rule; floating fine nodes contribute nothing."""
    T, W, H = inst.T, inst.W, inst.H
    Wc, Hc = (W + 1) // 2, (H + 1) // 2
    fl = network.floating_mask(inst).reshape(T, H, W)
    gx = np.zeros((T, Hc, max(Wc - 1, 0)))
    gy = np.zeros((T, max(Hc - 1, 0), Wc))
    for t in range(T):
        for y in range(H):
            for x in range(W):
                if fl[t, y, x]:
                    continue
                if x % 2 == 1 and x + 1 < W:   # crosses from aggregate x//2 to x//2 + 1
                    gx[t, y // 2, x // 2] += inst.gx[t, y, x]
                if y % 2 == 1 and y + 1 < H:
                    gy[t, y // 2, x // 2] += inst.gy[t, y, x]
    tsv, pads = {}, {}
    for t, x, y, g in zip(inst.tsv_tier, inst.tsv_x, inst.tsv_y, inst.tsv_g):
        if not fl[t, y, x]:
            key = (int(t), int(x) // 2, int(y) // 2)
            tsv[key] = tsv.get(key, 0.0) + g
    for t, x, y, g in zip(inst.pad_tier, inst.pad_x, inst.pad_y, inst.pad_g):
        if not fl[t, y, x]:
            key = (int(t), int(x) // 2, int(y) // 2)
            pads[key] = pads.get(key, 0.0) + g
    with np.errstate(divide="ignore"):
        rx = np.where(gx > 0, 1.0 / np.where(gx > 0, gx, 1.0), np.inf)
        ry = np.where(gy > 0, 1.0 / np.where(gy > 0, gy, 1.0), np.inf)
    return I.from_resistances(rx, ry, [(t, x, y, 1.0 / g) for (t, x, y), g in sorted(tsv.items())],
                              [(t, x, y, 1.0 / g) for (t, x, y), g in sorted(pads.items())], "coarse")


def galerkin(inst):
    """P^T G P over the coarse node ids (rows of aggregates without non-floating nodes are 0)."""
    T, W, H = inst.T, inst.W, inst.H
    Wc, Hc = (W + 1) // 2, (H + 1) // 2
    G = network.conductance_matrix(inst).toarray()
    fl = network.floating_mask(inst)
    P = np.zeros((inst.n, T * Hc * Wc))
    for t in range(T):
        for y in range(H):
            for x in range(W):
                i = (t * H + y) * W + x
                if not fl[i]:
                    P[i, (t * Hc + y // 2) * Wc + x // 2] = 1.0
    return P.T @ G @ P
