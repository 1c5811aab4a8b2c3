"""TSV-planning sweep: band-like against uniformly distributed TSV placements (paper Sec. IV-B).

The paper compares two TSV plans for the same load: all TSVs clustered in a central band
(as in HBM stacks) and TSVs spread uniformly over the die, and reports how many bumps
carry 95% of the total current (23.4% against 53.2% on its floorplan, which is not
available).  This module reproduces the method on synthetic early-stage floorplans:

  * floorplans: T uniform tiers (x/y segment resistance per tier), bumps (pads) on tier 0
    on a regular pitch, four functional blocks on the top tier drawing a uniform current
    density, and a TSV plan -- a central band of `band_rows` rows or a uniform grid, with
    the same number of through-stack TSV columns;
  * per plan, the library computes (all on the GPU): the all-node R map (the batching form,
    one shared launch per pass for every plan of the sweep), the exact IR drop of the load
    (er_solve with the block currents as right-hand sides) and the through-bump currents
    (er_pad_currents); the host then reads off the summary statistics.

Only inputs are drawn here; all arithmetic of the analysis runs in liber.so.
"""
from __future__ import annotations

import time

import numpy as np

from . import instances as I


def tsv_plan(W, H, count, pattern, band_rows=32):
    """(xs, ys) of `count` TSV columns.  'uniform': a regular grid over the whole die;
    'band': a regular grid inside the central band of `band_rows` rows."""
    if pattern == "uniform":
        y0, h = 0, H
    elif pattern == "band":
        h = min(band_rows, H)
        y0 = (H - h) // 2
    else:
        raise ValueError(pattern)
    # a grid of ny rows x nx columns with nx / ny close to W / h
    ny = max(1, int(round(np.sqrt(count * h / W))))
    ny = min(ny, h)
    nx = -(-count // ny)
    if nx > W:
        raise ValueError("too many TSVs for the region")
    xs = np.floor((np.arange(nx) + 0.5) * W / nx).astype(np.int32)
    ys = y0 + np.floor((np.arange(ny) + 0.5) * h / ny).astype(np.int32)
    gx, gy = np.meshgrid(xs, ys)
    return gx.ravel()[:count], gy.ravel()[:count]


def blocks(W, H, bw=None, bh=None):
    """Four functional blocks (x0, y0, width, height), one per die quadrant; 2:1 aspect
    like the paper's 2.35 x 1.18 mm^2 blocks."""
    bw = bw or W // 4
    bh = bh or H // 8
    cx = [W // 4, 3 * W // 4]
    cy = [H // 4, 3 * H // 4]
    return [(x - bw // 2, y - bh // 2, bw, bh) for y in cy for x in cx]


def floorplan(pattern, n_tsv=1024, T=4, W=256, H=256, band_rows=32, r_tier=(0.05, 0.1, 0.1, 0.05),
              r_tsv=0.02, pad_pitch=8, r_pad=0.01):
    """One plan as a network instance (uniform tiers, through-stack TSV columns, pads on tier 0)."""
    xs, ys = tsv_plan(W, H, n_tsv, pattern, band_rows)
    r = np.resize(np.asarray(r_tier, dtype=np.float64), T)
    inst = I.uniform(T, W, H, r, r, tsv=I._columns(T, xs, ys, np.full(len(xs), r_tsv)),
                     pads=I._pads_on_pitch(W, H, pad_pitch, r_pad), name=f"plan_{pattern}_{n_tsv}")
    inst.meta.update({"pattern": pattern, "n_tsv": int(n_tsv), "band_rows": int(band_rows)})
    return inst


def block_loads(inst, current_per_block=1.0):
    """(load node ids [L], currents [L][4]): column b draws `current_per_block` amperes spread
    uniformly over block b's nodes on the top tier (one scenario per block; superposition
    gives any combination)."""
    nodes, cur = [], []
    top = (inst.T - 1) * inst.W * inst.H
    for b, (x0, y0, bw, bh) in enumerate(blocks(inst.W, inst.H)):
        yy, xx = np.meshgrid(np.arange(y0, y0 + bh), np.arange(x0, x0 + bw), indexing="ij")
        ids = top + yy.ravel() * inst.W + xx.ravel()
        c = np.zeros((len(ids), 4))
        c[:, b] = current_per_block / len(ids)
        nodes.append(ids)
        cur.append(c)
    return np.concatenate(nodes).astype(np.int64), np.concatenate(cur)


def bump_share(currents, share=0.95):
    """Fraction of bumps that together carry `share` of the total current, largest first."""
    mag = np.abs(np.asarray(currents, dtype=np.float64))
    if not mag.sum() > 0:
        return 0.0  # no current: no bump is needed to carry any share of it
    need = share * mag.sum() * (1 - 1e-12)
    acc, used = 0.0, 0
    for c in sorted(mag, reverse=True):
        if acc >= need and used > 0:
            break
        acc += c
        used += 1
    return used / max(len(mag), 1)


def sweep(plans, k=64, seed=1, prec="fp32", device=None):
    """Analyse every plan: R maps of all plans in one batching-form call, then per plan the
    exact IR drop of the four block loads (er_solve, 4 right-hand sides) and the through-bump
    currents of the total load.  Returns one dict per plan and the timings."""
    import torch

    from . import er

    dev = device or torch.device("cuda", torch.cuda.current_device())
    t0 = time.perf_counter()
    grids = [er.grid_create(p) for p in plans]
    Rmaps = [torch.empty(p.n, dtype=torch.float64, device=dev) for p in plans]
    er.batch_solve(grids, k, seed, Rmaps, prec=prec)
    torch.cuda.synchronize()
    t_maps = time.perf_counter() - t0
    out = []
    dt = torch.float32 if prec == "fp32" else torch.float64
    t1 = time.perf_counter()
    for p, g, Rm in zip(plans, grids, Rmaps):
        loads, cur = block_loads(p)
        B = np.zeros((p.n, 4))
        np.add.at(B, loads, cur)
        Bd = torch.from_numpy(B).to(dev, dt)
        V = torch.empty_like(Bd)
        er.solve(g, Bd, V, 4, prec)
        Ip = torch.empty((len(p.pad_g), 4), dtype=torch.float64, device=dev)
        er.pad_currents(g, V, 4, prec, Ip)
        torch.cuda.synchronize()
        vload = V.cpu().numpy().astype(np.float64)[loads].sum(axis=1)  # total load: superposition
        rload = Rm.cpu().numpy()[loads]
        ip = Ip.cpu().numpy().sum(axis=1)
        out.append({"pattern": p.meta.get("pattern"), "n_tsv": p.meta.get("n_tsv"),
                    "band_rows": p.meta.get("band_rows"),
                    "bump_share_95": bump_share(ip), "pad_current_sum": float(ip.sum()),
                    "load_current": float(cur.sum()), "max_ir_drop_at_loads": float(vload.max()),
                    "max_R_at_loads": float(rload.max()), "mean_R_at_loads": float(rload.mean())})
    t_exact = time.perf_counter() - t1
    for g in grids:
        g.destroy()
    return out, {"maps_s": t_maps, "exact_s": t_exact}
