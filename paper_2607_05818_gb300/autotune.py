"""Autotuner for the launch shape of the solve's stencil kernels, per network size class.

For a size class (tiers, width, height, k, precision, preconditioner) it times a few PCG
iterations through the C ABI for each candidate, with the library's own per-pass CUDA-event
timing (er_solve_opts.profile), and keeps the fastest:
  - Jacobi: the y rows swept by one CTA of the stencil passes (best_rows);
  - multigrid: the launch order of the tiled V-cycle and CG kernels, the RHS column blocks of
    a tile adjacent or outermost (best_mg_order).  The order decides which CTAs share L2 lines,
    not the arithmetic, so the tuned solve gives bitwise the map of the untuned one.
Results are cached in a JSON file (ER_AUTOTUNE_CACHE, default ~/.cache/er3d_autotune.json),
keyed by the size class, so each class is measured once per machine.
"""
from __future__ import annotations

import json
import os
import threading

CANDIDATE_ROWS = (16, 32, 64, 128)
CANDIDATE_MG_ORDERS = (1, 2)  # er_solve_opts.block_order: column blocks adjacent, outermost
_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("ER_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "er3d_autotune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def key(inst, k: int, prec: str) -> str:
    return f"{inst.T}x{inst.W}x{inst.H}_k{k}_{prec}"


def measure(inst, k: int, prec: str = "fp32", iters: int = 8, rows_list=CANDIDATE_ROWS) -> dict:
    """Per-iteration pass time (ms) for each candidate row count on this network."""
    import torch

    from . import er
    g = er.grid_create(inst)
    dt = torch.float32 if prec == "fp32" else torch.float64
    Y = torch.empty((inst.n, k), dtype=dt, device="cuda")
    Z = torch.empty_like(Y)
    er.sketch(g, k, 1, prec, Y)
    out = {}
    for rows in rows_list:
        if rows > inst.H and rows != rows_list[0]:
            continue
        best = None
        for _ in range(2):
            o = er.default_solve_opts(prec, maxit=iters, profile=1, tile_rows=rows, replace_every=10 ** 6)
            _, st = er.solve(g, Y, Z, k, prec, o, allow_unconverged=True)
            t = (st["kernel_ms"][er.PASS_A] + st["kernel_ms"][er.PASS_B] + st["kernel_ms"][er.PASS_B0]) / max(
                st["iterations"], 1)
            best = t if best is None else min(best, t)
        out[rows] = best
    g.destroy()
    return out


def best_rows(inst, k: int, prec: str = "fp32") -> int:
    """The cached best row count for this size class, measuring it on first use."""
    kk = key(inst, k, prec)
    with _lock:
        d = _load()
        if kk in d:
            return int(d[kk]["rows"])
        times = measure(inst, k, prec)
        rows = min(times, key=times.get)
        d[kk] = {"rows": int(rows), "ms_per_iteration": {str(r): t for r, t in times.items()}}
        _store(d)
        return int(rows)


def measure_mg(inst, k: int, iters: int = 6, orders=CANDIDATE_MG_ORDERS) -> dict:
    """Per-iteration kernel time (ms) of the multigrid solve for each candidate launch order."""
    import torch

    from . import er
    g = er.grid_create(inst)
    Y = torch.empty((inst.n, k), dtype=torch.float32, device="cuda")
    Z = torch.empty_like(Y)
    er.sketch(g, k, 1, "fp32", Y)
    out = {}
    for order in orders:
        best = None
        for _ in range(2):
            o = er.default_solve_opts("fp32", precond=1, maxit=iters, profile=1, block_order=order,
                                      replace_every=10 ** 6)
            _, st = er.solve(g, Y, Z, k, "fp32", o, allow_unconverged=True)
            t = sum(st["kernel_ms"]) / max(st["iterations"], 1)
            best = t if best is None else min(best, t)
        out[order] = best
    g.destroy()
    return out


def best_mg_order(inst, k: int) -> int:
    """The cached best launch order (er_solve_opts.block_order) of the multigrid kernels for
    this size class."""
    kk = key(inst, k, "fp32") + "_mg"
    with _lock:
        d = _load()
        if kk in d:
            return int(d[kk]["order"])
        times = measure_mg(inst, k)
        order = min(times, key=times.get)
        d[kk] = {"order": int(order), "ms_per_iteration": {str(r): t for r, t in times.items()}}
        _store(d)
        return int(order)
