"""Thin ctypes binding of liber.so (argument marshalling only).

Every call goes straight to the C ABI declared in include/er.h; all arithmetic runs
in the library's CUDA kernels.  PyTorch is used only to hand over device memory and
the current CUDA stream.  Importing this module loads the shared library and raises
ImportError if it has not been built (``__graft_entry__.build()``): there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int32, c_int64, c_uint64, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "liber.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")

_lib = ctypes.CDLL(LIB_PATH)

ER_OK, ER_ERR_INVALID_ARG, ER_ERR_CUDA, ER_ERR_OOM, ER_ERR_NO_SUPPLY, ER_ERR_NOT_CONVERGED, \
    ER_ERR_TIMEOUT, ER_WARN_FLOATING = range(8)
ER_FP64, ER_FP32_REFINE = 0, 1
PRECISIONS = {"fp64": ER_FP64, "fp32": ER_FP32_REFINE, ER_FP64: ER_FP64, ER_FP32_REFINE: ER_FP32_REFINE}


class er_tier(ctypes.Structure):
    _fields_ = [("W", c_int32), ("H", c_int32), ("gx", c_void_p), ("gy", c_void_p)]


class er_tsv(ctypes.Structure):
    _fields_ = [("tier", c_int32), ("x", c_int32), ("y", c_int32), ("g", c_double)]


class er_pad(ctypes.Structure):
    _fields_ = [("tier", c_int32), ("x", c_int32), ("y", c_int32), ("g", c_double)]


class er_options(ctypes.Structure):
    _fields_ = [("device", c_int32), ("reserved", c_int32 * 7)]


class er_solve_opts(ctypes.Structure):
    _fields_ = [("tol", c_double), ("maxit", c_int32), ("check_every", c_int32),
                ("replace_every", c_int32), ("use_graph", c_int32),
                ("profile", c_int32), ("tile_rows", c_int32), ("block_order", c_int32),
                ("precond", c_int32)]


class er_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", c_int32), ("sweeps", c_int32), ("converged_cols", c_int32),
                ("k", c_int32), ("max_rel_residual", c_double), ("seconds", c_double),
                ("launches", c_int32 * 8), ("kernel_ms", c_double * 8)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["launches"] = list(self.launches)
        d["kernel_ms"] = list(self.kernel_ms)
        return d


PASS_A, PASS_B, PASS_R, PASS_OTHER, PASS_B0, PASS_MG, PASS_MG_DOWN, PASS_MG_UP = range(8)


class er_batch_stats(ctypes.Structure):
    _fields_ = [("n_grids", c_int32), ("iterations", c_int32), ("replacements", c_int32),
                ("converged", c_int32), ("nodes", c_int64), ("max_rel_residual", c_double),
                ("seconds", c_double), ("launches", c_int32), ("graph_captures", c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class er_stack(ctypes.Structure):
    _fields_ = [("M", c_int32), ("N", c_int32), ("d", c_int32), ("p", c_int32), ("r", c_void_p), ("s", c_void_p),
                ("tsv_xy", c_void_p), ("Rt", c_void_p)]


class er_stack_stats(ctypes.Structure):
    _fields_ = [("n_system", c_int32), ("wu_pairs", c_int64), ("ms_wu", c_double), ("ms_build", c_double),
                ("ms_lu", c_double), ("ms_solve", c_double), ("ms_dot", c_double), ("seconds", c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class er_unet_shape(ctypes.Structure):
    _fields_ = [("in_ch", c_int32), ("out_ch", c_int32), ("levels", c_int32), ("base", c_int32), ("H", c_int32),
                ("W", c_int32)]


class er_conv_info(ctypes.Structure):
    _fields_ = [("kernel", c_int32), ("tile_n", c_int32), ("k_step", c_int32), ("reserved", c_int32)]

    def as_dict(self):
        return {"kernel": {1: "tma", 2: "staged"}.get(self.kernel, self.kernel), "tile_n": self.tile_n,
                "k_step": self.k_step}


_S = c_int32  # er_status
_sig = {
    "er_default_solve_opts": (er_solve_opts, [c_int32]),
    "er_grid_create": (_S, [POINTER(er_tier), c_int32, POINTER(er_tsv), c_int64, POINTER(er_pad), c_int64,
                            POINTER(er_options), c_void_p, POINTER(c_void_p)]),
    "er_grid_destroy": (_S, [c_void_p]),
    "er_grid_info": (_S, [c_void_p, POINTER(c_int64), POINTER(c_int64), POINTER(c_int64), POINTER(c_int64)]),
    "er_sketch": (_S, [c_void_p, c_int32, c_uint64, c_int32, c_void_p, c_void_p]),
    "er_sketch_cols": (_S, [c_void_p, c_int32, c_int32, c_int32, c_uint64, c_int32, c_void_p, c_void_p]),
    "er_solve": (_S, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, POINTER(er_solve_opts),
                      POINTER(er_solve_stats), c_void_p]),
    "er_solve_noalloc": (_S, [c_void_p, c_void_p, c_void_p, c_int32, POINTER(er_solve_opts),
                              POINTER(er_solve_stats), c_void_p]),
    "er_reff_map": (_S, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p]),
    "er_batch_solve": (_S, [POINTER(c_void_p), c_int32, c_int32, c_uint64, c_int32, POINTER(c_int32),
                            POINTER(c_void_p), POINTER(er_solve_opts), POINTER(er_batch_stats), c_void_p]),
    "er_reff_map_host": (_S, [POINTER(er_tier), c_int32, POINTER(er_tsv), c_int64, POINTER(er_pad), c_int64,
                              c_int32, c_uint64, c_int32, POINTER(er_solve_opts), c_void_p,
                              POINTER(er_solve_stats), c_void_p]),
    "er_release_pool": (_S, []),
    "er_pair_reff": (_S, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_int32, c_void_p, c_int32, c_void_p,
                          c_void_p]),
    "er_ir_drop": (_S, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_int64, c_int32, c_void_p,
                        c_void_p]),
    "er_surrogate_create": (_S, [POINTER(er_unet_shape), c_uint64, POINTER(c_void_p)]),
    "er_surrogate_destroy": (_S, [c_void_p]),
    "er_surrogate_num_params": (_S, [c_void_p, POINTER(c_int64)]),
    "er_surrogate_get_params": (_S, [c_void_p, c_void_p, c_int64]),
    "er_surrogate_set_params": (_S, [c_void_p, c_void_p, c_int64]),
    "er_surrogate_infer": (_S, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "er_surrogate_grad": (_S, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p, POINTER(c_double),
                               c_void_p]),
    "er_surrogate_train_step": (_S, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, ctypes.c_float,
                                     POINTER(c_double), c_void_p]),
    "er_surrogate_set_tile_n": (_S, [c_void_p, c_int32]),
    "er_conv3x3_forward": (_S, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32,
                                c_int32, c_void_p, POINTER(er_conv_info), c_void_p]),
    "er_conv3x3_dgrad": (_S, [c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_int32,
                              c_void_p, POINTER(er_conv_info), c_void_p]),
    "er_conv3x3_wgrad": (_S, [c_void_p, c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p]),
    "er_conv_launch_counts": (_S, [POINTER(c_int64), c_int32, c_int32]),
    "er_pad_currents": (_S, [c_void_p, c_void_p, c_int32, c_int32, c_void_p, c_void_p]),
    "er_stack_pairs": (_S, [POINTER(er_stack), c_void_p, c_int32, c_void_p, c_int32, c_void_p,
                            POINTER(er_stack_stats), c_void_p]),
    "er_status_str": (ctypes.c_char_p, [c_int32]),
    "er_last_error": (ctypes.c_char_p, []),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class ErError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.er_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_lib.er_status_str(status).decode()} ({msg})")


def _check(status, where, ok=(ER_OK, ER_WARN_FLOATING)):
    if status not in ok:
        raise ErError(status, where)
    return status


def status_str(s) -> str:
    return _lib.er_status_str(s).decode()


def default_solve_opts(prec="fp64", **over) -> er_solve_opts:
    o = _lib.er_default_solve_opts(PRECISIONS[prec])
    for k, v in over.items():
        setattr(o, k, v)
    return o


# ------------------------------------------------------------------ marshalling

_SEG = np.dtype([("tier", "<i4"), ("x", "<i4"), ("y", "<i4"), ("g", "<f8")], align=True)
assert _SEG.itemsize == ctypes.sizeof(er_tsv) == ctypes.sizeof(er_pad)


class _Marshalled:
    """ctypes views of one network instance (keeps the numpy buffers alive)."""

    def __init__(self, inst):
        T, W, H = inst.T, inst.W, inst.H
        self.gx = [np.ascontiguousarray(inst.gx[t], dtype=np.float64) for t in range(T)]
        self.gy = [np.ascontiguousarray(inst.gy[t], dtype=np.float64) for t in range(T)]
        self.tiers = (er_tier * T)()
        for t in range(T):
            self.tiers[t].W, self.tiers[t].H = W, H
            self.tiers[t].gx = self.gx[t].ctypes.data if self.gx[t].size else None
            self.tiers[t].gy = self.gy[t].ctypes.data if self.gy[t].size else None
        self.nt, self.npd = len(inst.tsv_g), len(inst.pad_g)
        self._tsv = self._segments(inst.tsv_tier, inst.tsv_x, inst.tsv_y, inst.tsv_g)
        self._pads = self._segments(inst.pad_tier, inst.pad_x, inst.pad_y, inst.pad_g)
        self.tsv = ctypes.cast(self._tsv.ctypes.data, POINTER(er_tsv))
        self.pads = ctypes.cast(self._pads.ctypes.data, POINTER(er_pad))
        self.T = T

    @staticmethod
    def _segments(tier, x, y, g):
        a = np.zeros(max(len(g), 1), dtype=_SEG)
        if len(g):
            a["tier"], a["x"], a["y"], a["g"] = tier, x, y, g
        return a


def _ptr(t) -> int:
    """Device pointer of a torch tensor (or an int address)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Grid:
    """An er_grid handle (device-resident network)."""

    def __init__(self, inst, device: int = -1, stream=None):
        m = _Marshalled(inst)
        opt = er_options()
        opt.device = device
        h = c_void_p()
        self.status = _check(_lib.er_grid_create(m.tiers, m.T, m.tsv, m.nt, m.pads, m.npd, ctypes.byref(opt),
                                                 _stream(stream), ctypes.byref(h)), "er_grid_create")
        self.handle = h
        self.T, self.W, self.H = inst.T, inst.W, inst.H

    def info(self):
        n, f, e, b = c_int64(), c_int64(), c_int64(), c_int64()
        _check(_lib.er_grid_info(self.handle, ctypes.byref(n), ctypes.byref(f), ctypes.byref(e), ctypes.byref(b)),
               "er_grid_info")
        return {"n_nodes": n.value, "n_floating": f.value, "n_edges": e.value, "h2d_bytes": b.value}

    def destroy(self):
        if getattr(self, "handle", None):
            _lib.er_grid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def grid_create(inst, device: int = -1, stream=None) -> Grid:
    return Grid(inst, device, stream)


def sketch(grid: Grid, k: int, seed: int, prec, Yt, stream=None):
    return _check(_lib.er_sketch(grid.handle, k, c_uint64(seed), PRECISIONS[prec], _ptr(Yt), _stream(stream)),
                  "er_sketch")


def sketch_cols(grid: Grid, k_total: int, j0: int, k_local: int, seed: int, prec, Yt, stream=None):
    """Columns j0 .. j0 + k_local - 1 of the k_total-column sketch into Yt [n][k_local]."""
    return _check(_lib.er_sketch_cols(grid.handle, k_total, j0, k_local, c_uint64(seed), PRECISIONS[prec], _ptr(Yt),
                                      _stream(stream)), "er_sketch_cols")


def column_shard(k: int, world: int, rank: int) -> tuple[int, int]:
    """(j0, k_local) of rank's share of k sketch columns over `world` ranks: contiguous, disjoint,
    covering 0 .. k-1, each a multiple of 4 columns (the last ranks may get 4 fewer)."""
    if k % 4 or k < 4 * world:
        raise ValueError("k must be a multiple of 4 with at least 4 columns per rank")
    q = k // 4
    base, extra = divmod(q, world)
    j0 = 4 * (rank * base + min(rank, extra))
    return j0, 4 * (base + (1 if rank < extra else 0))


def solve(grid: Grid, Yt, Z, k: int, prec, opts: er_solve_opts | None = None, stream=None, allow_unconverged=False):
    st = er_solve_stats()
    ok = (ER_OK, ER_ERR_NOT_CONVERGED) if allow_unconverged else (ER_OK,)
    s = _lib.er_solve(grid.handle, _ptr(Yt), _ptr(Z), k, PRECISIONS[prec],
                      ctypes.byref(opts) if opts is not None else None, ctypes.byref(st), _stream(stream))
    _check(s, "er_solve", ok)
    return s, st.as_dict()


def solve_noalloc(grid: Grid, Yt, Z, k: int, opts: er_solve_opts | None = None, stream=None,
                  allow_unconverged=False):
    """FP64 solve whose workspace is a fixed static device array (no device allocation)."""
    st = er_solve_stats()
    ok = (ER_OK, ER_ERR_NOT_CONVERGED) if allow_unconverged else (ER_OK,)
    s = _lib.er_solve_noalloc(grid.handle, _ptr(Yt), _ptr(Z), k,
                              ctypes.byref(opts) if opts is not None else None, ctypes.byref(st), _stream(stream))
    _check(s, "er_solve_noalloc", ok)
    return s, st.as_dict()


def reff_map(grid: Grid, Z, k: int, prec, R, stream=None):
    return _check(_lib.er_reff_map(grid.handle, _ptr(Z), k, PRECISIONS[prec], _ptr(R), _stream(stream)),
                  "er_reff_map")


def pair_reff(grid: Grid, Z, k: int, prec, u, v, Rp, stream=None):
    """Rp[a, b] = ||Z_u[a] - Z_v[b]||^2 (device FP64 [len(u)][len(v)]); u, v: host node ids."""
    ua = np.ascontiguousarray(u, dtype=np.int64)
    va = np.ascontiguousarray(v, dtype=np.int64)
    return _check(_lib.er_pair_reff(grid.handle, _ptr(Z), k, PRECISIONS[prec], ua.ctypes.data, len(ua),
                                    va.ctypes.data, len(va), _ptr(Rp), _stream(stream)), "er_pair_reff")


def ir_drop(grid: Grid, Z, k: int, prec, loads, currents, drop, stream=None):
    """drop (device FP64 [n][S]) = Z (Z^T I) for host loads [L] and currents [L] or [L][S]."""
    la = np.ascontiguousarray(loads, dtype=np.int64)
    cur = np.asarray(currents, dtype=np.float64)
    cur = np.ascontiguousarray(cur[:, None] if cur.ndim == 1 else cur)
    if cur.shape[0] != len(la):
        raise ValueError("currents must have one row per load")
    return _check(_lib.er_ir_drop(grid.handle, _ptr(Z), k, PRECISIONS[prec], la.ctypes.data, cur.ctypes.data,
                                  len(la), cur.shape[1], _ptr(drop), _stream(stream)), "er_ir_drop")


def pad_currents(grid: Grid, V, S: int, prec, I_pad, stream=None):
    """I_pad (device FP64 [n_pads][S]) = g_pad * V at each pad's node; V device [n][S]."""
    return _check(_lib.er_pad_currents(grid.handle, _ptr(V), S, PRECISIONS[prec], _ptr(I_pad), _stream(stream)),
                  "er_pad_currents")


def stack_pairs(M, N, r, s, tsv_xy, Rt, bumps, loads, R, stream=None):
    """Bump-to-load effective resistances of a uniform die stack by the paper's reduced TSV
    system.  r, s: [d]; tsv_xy: [p][2]; Rt: [d-1][p]; bumps [m][2] (die 0), loads [n][2]
    (die d-1), host arrays; R: device FP64 [m][n].  Returns the phase statistics."""
    r_ = np.ascontiguousarray(r, dtype=np.float64)
    s_ = np.ascontiguousarray(s, dtype=np.float64)
    t_ = np.ascontiguousarray(tsv_xy, dtype=np.int32).reshape(-1, 2)
    Rt_ = np.ascontiguousarray(Rt, dtype=np.float64).reshape(len(r_) - 1, len(t_))
    b_ = np.ascontiguousarray(bumps, dtype=np.int32).reshape(-1, 2)
    l_ = np.ascontiguousarray(loads, dtype=np.int32).reshape(-1, 2)
    st = er_stack(M, N, len(r_), len(t_), r_.ctypes.data, s_.ctypes.data, t_.ctypes.data, Rt_.ctypes.data)
    stats = er_stack_stats()
    _check(_lib.er_stack_pairs(ctypes.byref(st), b_.ctypes.data, len(b_), l_.ctypes.data, len(l_), _ptr(R),
                               ctypes.byref(stats), _stream(stream)), "er_stack_pairs")
    return stats.as_dict()


def batch_solve(grids, k: int, seed: int, R_out, prec="fp32", opts: er_solve_opts | None = None,
                tile_rows=None, stream=None, allow_unconverged=False):
    """Batching form: R maps of many networks; network c uses seed + c.  With opts.precond 0
    (Jacobi) every pass is one shared launch over all networks; with precond 1 every pass of the
    multigrid iteration is one persistent launch over all running networks and the loop is a
    device-side conditional graph node.  R_out: list of device FP64 tensors (one per grid)."""
    n = len(grids)
    hs = (c_void_p * n)(*[g.handle.value if isinstance(g.handle, c_void_p) else g.handle for g in grids])
    rs = (c_void_p * n)(*[_ptr(r) for r in R_out])
    tr = (c_int32 * n)(*tile_rows) if tile_rows is not None else None
    st = er_batch_stats()
    ok = (ER_OK, ER_ERR_NOT_CONVERGED) if allow_unconverged else (ER_OK,)
    s = _lib.er_batch_solve(hs, n, k, c_uint64(seed), PRECISIONS[prec], tr, rs,
                            ctypes.byref(opts) if opts is not None else None, ctypes.byref(st), _stream(stream))
    _check(s, "er_batch_solve", ok)
    return s, st.as_dict()


def reff_map_host(inst, k: int, seed: int, prec, opts: er_solve_opts | None = None, R_host=None, stream=None,
                  allow_unconverged=False):
    """Host instance in, host R map (numpy FP64) out; copies run inside the library call."""
    m = _Marshalled(inst)
    R = np.empty(inst.T * inst.W * inst.H, dtype=np.float64) if R_host is None else R_host
    st = er_solve_stats()
    ok = (ER_OK, ER_WARN_FLOATING, ER_ERR_NOT_CONVERGED) if allow_unconverged else (ER_OK, ER_WARN_FLOATING)
    s = _lib.er_reff_map_host(m.tiers, m.T, m.tsv, m.nt, m.pads, m.npd, k, c_uint64(seed), PRECISIONS[prec],
                              ctypes.byref(opts) if opts is not None else None,
                              R.ctypes.data if isinstance(R, np.ndarray) else _ptr(R), ctypes.byref(st),
                              _stream(stream))
    _check(s, "er_reff_map_host", ok)
    return R, st.as_dict()


class Surrogate:
    """An er_surrogate handle: the BF16 U-Net from per-node maps to log R."""

    def __init__(self, in_ch=32, out_ch=4, levels=6, base=32, H=256, W=256, seed=1):
        self.shape = er_unet_shape(in_ch, out_ch, levels, base, H, W)
        h = c_void_p()
        _check(_lib.er_surrogate_create(ctypes.byref(self.shape), c_uint64(seed), ctypes.byref(h)),
               "er_surrogate_create")
        self.handle = h
        self._steps = 0

    def step_count(self) -> int:
        """Adam steps taken through this handle."""
        return self._steps

    def num_params(self) -> int:
        n = c_int64()
        _check(_lib.er_surrogate_num_params(self.handle, ctypes.byref(n)), "er_surrogate_num_params")
        return n.value

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params(), dtype=np.float32)
        _check(_lib.er_surrogate_get_params(self.handle, out.ctypes.data, out.size), "er_surrogate_get_params")
        return out

    def set_params(self, flat) -> None:
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(_lib.er_surrogate_set_params(self.handle, a.ctypes.data, a.size), "er_surrogate_set_params")

    def infer(self, maps, B, out, stream=None):
        _check(_lib.er_surrogate_infer(self.handle, _ptr(maps), B, _ptr(out), _stream(stream)), "er_surrogate_infer")

    def grad(self, maps, target, mask, B, stream=None):
        g = np.empty(self.num_params(), dtype=np.float32)
        loss = c_double()
        _check(_lib.er_surrogate_grad(self.handle, _ptr(maps), _ptr(target), _ptr(mask), B, g.ctypes.data,
                                      ctypes.byref(loss), _stream(stream)), "er_surrogate_grad")
        return loss.value, g

    def train_step(self, maps, target, mask, B, lr, stream=None) -> float:
        loss = c_double()
        _check(_lib.er_surrogate_train_step(self.handle, _ptr(maps), _ptr(target), _ptr(mask), B, ctypes.c_float(lr),
                                            ctypes.byref(loss), _stream(stream)), "er_surrogate_train_step")
        self._steps += 1
        return loss.value

    def set_tile_n(self, tile_n: int) -> None:
        _check(_lib.er_surrogate_set_tile_n(self.handle, int(tile_n)), "er_surrogate_set_tile_n")

    def destroy(self):
        if getattr(self, "handle", None):
            _lib.er_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def conv3x3_forward(x, w, bias, B, H, W, cin, cout, y, relu=True, tile_n=0, stream=None) -> dict:
    """One surrogate convolution layer: x, y BF16 [B][H][W][c] device tensors, w FP32
    [cout][3][3][cin], bias FP32 [cout] or None.  Returns what ran."""
    info = er_conv_info()
    _check(_lib.er_conv3x3_forward(_ptr(x), _ptr(w), _ptr(bias), B, H, W, cin, cout, int(bool(relu)), tile_n, _ptr(y),
                                   ctypes.byref(info), _stream(stream)), "er_conv3x3_forward")
    return info.as_dict()


def conv3x3_dgrad(dy, w, x, B, H, W, cin, cout, dx, tile_n=0, stream=None) -> dict:
    """Data gradient of that layer through the ReLU of its input x."""
    info = er_conv_info()
    _check(_lib.er_conv3x3_dgrad(_ptr(dy), _ptr(w), _ptr(x), B, H, W, cin, cout, tile_n, _ptr(dx),
                                 ctypes.byref(info), _stream(stream)), "er_conv3x3_dgrad")
    return info.as_dict()


def conv3x3_wgrad(x, dy, B, H, W, cin, cout, dw, stream=None) -> None:
    """Weight gradient of that layer into dw (FP32 [cout][3][3][cin], overwritten)."""
    _check(_lib.er_conv3x3_wgrad(_ptr(x), _ptr(dy), B, H, W, cin, cout, _ptr(dw), _stream(stream)), "er_conv3x3_wgrad")


CONV_COUNT_SLOTS = ([f"tma_k32_n{n}" for n in (32, 64, 96, 128, 192, 256)]
                    + [f"tma_k64_n{n}" for n in (32, 64, 96, 128, 192, 256)] + ["staged", "wgrad_mma", "wgrad_tc", "-"])


def conv_launch_counts(reset=False) -> dict:
    """Launches of the convolution kernels since the last reset, by kernel, K step and N tile."""
    a = (c_int64 * 16)()
    _check(_lib.er_conv_launch_counts(a, 16, int(bool(reset))), "er_conv_launch_counts")
    return {name: int(v) for name, v in zip(CONV_COUNT_SLOTS, a) if name != "-"}


def release_pool():
    return _lib.er_release_pool()


def exported_symbols():
    return sorted(_sig)
