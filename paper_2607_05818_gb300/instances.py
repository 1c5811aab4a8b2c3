"""Seeded synthetic 3D-IC power-delivery-network instances.

This module only draws inputs: per-segment wire conductances of each tier mesh,
TSV segments between adjacent tiers and pad conductances to the ideal supply.
It holds none of the effective-resistance arithmetic, so both the CUDA path and
the CPU oracle may take their inputs from it.

Model (paper Sec. III-B, Table "Notations"): every tier is a W x H resistive
mesh; a TSV is a through-stack column that meets every die at the same (x, y)
and contributes one segment per adjacent tier pair (Rt_k^{i,i+1}); bumps/pads
tie mesh nodes to an ideal supply.  Node id i = (t*H + y)*W + x (tier-major,
x fastest).

Arrays (all float64 conductances in siemens, 0 = open segment):
  gx[t, y, x]   segment (t,y,x)-(t,y,x+1), shape (T, H, W-1)
  gy[t, y, x]   segment (t,y,x)-(t,y+1,x), shape (T, H-1, W)
  tsv_*         segment (tier,x,y)-(tier+1,x,y), conductance tsv_g
  pad_*         node (tier,x,y) to the supply, conductance pad_g
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20260701


@dataclass
class Instance:
    T: int
    W: int
    H: int
    gx: np.ndarray
    gy: np.ndarray
    tsv_tier: np.ndarray
    tsv_x: np.ndarray
    tsv_y: np.ndarray
    tsv_g: np.ndarray
    pad_tier: np.ndarray
    pad_x: np.ndarray
    pad_y: np.ndarray
    pad_g: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.T * self.W * self.H

    def scaled(self, c: float) -> "Instance":
        """Same network with every resistance multiplied by c."""
        return Instance(self.T, self.W, self.H, self.gx / c, self.gy / c,
                        self.tsv_tier.copy(), self.tsv_x.copy(), self.tsv_y.copy(),
                        self.tsv_g / c, self.pad_tier.copy(), self.pad_x.copy(),
                        self.pad_y.copy(), self.pad_g / c, self.name + f"*{c}",
                        dict(self.meta))

    def validate(self) -> None:
        T, W, H = self.T, self.W, self.H
        assert self.gx.shape == (T, H, W - 1) and self.gy.shape == (T, H - 1, W)
        for a in (self.tsv_tier, self.tsv_x, self.tsv_y, self.tsv_g):
            assert a.shape == self.tsv_tier.shape
        for a in (self.pad_tier, self.pad_x, self.pad_y, self.pad_g):
            assert a.shape == self.pad_tier.shape
        assert np.all(self.gx >= 0) and np.all(self.gy >= 0)
        assert np.all(self.tsv_g > 0) and np.all(self.pad_g > 0)
        if len(self.tsv_tier):
            assert self.tsv_tier.min() >= 0 and self.tsv_tier.max() < T - 1
            assert self.tsv_x.min() >= 0 and self.tsv_x.max() < W
            assert self.tsv_y.min() >= 0 and self.tsv_y.max() < H
        if len(self.pad_tier):
            assert self.pad_tier.min() >= 0 and self.pad_tier.max() < T
            assert self.pad_x.min() >= 0 and self.pad_x.max() < W
            assert self.pad_y.min() >= 0 and self.pad_y.max() < H


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32).reshape(-1))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))


def from_resistances(rx, ry, tsv=(), pads=(), name="") -> Instance:
    """Build an instance from per-tier resistance arrays.

    rx: (T, H, W-1) x-segment resistances (np.inf = open); ry: (T, H-1, W).
    tsv: iterable of (tier, x, y, r); pads: iterable of (tier, x, y, r).
    """
    rx = np.asarray(rx, dtype=np.float64)
    ry = np.asarray(ry, dtype=np.float64)
    T, H, Wm1 = rx.shape
    W = Wm1 + 1
    assert ry.shape == (T, H - 1, W)
    with np.errstate(divide="ignore"):
        gx = np.where(np.isinf(rx), 0.0, 1.0 / rx)
        gy = np.where(np.isinf(ry), 0.0, 1.0 / ry)
    tsv = list(tsv)
    pads = list(pads)
    inst = Instance(
        T, W, H, gx, gy,
        _i32([t[0] for t in tsv]), _i32([t[1] for t in tsv]), _i32([t[2] for t in tsv]),
        _f64([1.0 / t[3] for t in tsv]),
        _i32([p[0] for p in pads]), _i32([p[1] for p in pads]), _i32([p[2] for p in pads]),
        _f64([1.0 / p[3] for p in pads]), name)
    inst.validate()
    return inst


def uniform(T, W, H, r, s, tsv=(), pads=(), name="uniform") -> Instance:
    """Uniform tiers: x-segments r[t], y-segments s[t] (scalars broadcast)."""
    r = np.broadcast_to(np.asarray(r, dtype=np.float64), (T,))
    s = np.broadcast_to(np.asarray(s, dtype=np.float64), (T,))
    rx = np.broadcast_to(r[:, None, None], (T, H, W - 1)).copy()
    ry = np.broadcast_to(s[:, None, None], (T, H - 1, W)).copy()
    return from_resistances(rx, ry, tsv, pads, name)


# --------------------------------------------------------------------------
# random pieces
# --------------------------------------------------------------------------

def _jittered(rng, base, shape, sigma):
    """Per-segment resistance base * lognormal(mu=0, sigma)."""
    if sigma > 0:
        return base * rng.lognormal(0.0, sigma, size=shape)
    return np.full(shape, float(base))


def _unique_positions(rng, W, H, count, draw):
    """Draw `count` distinct (x, y) with `draw(rng, m) -> (x, y)`; duplicates are redrawn."""
    taken = set()
    xs, ys = [], []
    need = count
    for _ in range(10000):
        if need == 0:
            break
        x, y = draw(rng, need)
        x = np.clip(np.rint(x), 0, W - 1).astype(np.int64)
        y = np.clip(np.rint(y), 0, H - 1).astype(np.int64)
        for a, b in zip(x, y):
            key = (int(a), int(b))
            if key not in taken:
                taken.add(key)
                xs.append(key[0])
                ys.append(key[1])
                need -= 1
                if need == 0:
                    break
    if need:
        raise ValueError("could not place TSVs without duplicates")
    return np.array(xs, dtype=np.int32), np.array(ys, dtype=np.int32)


def tsv_uniform_xy(rng, W, H, count):
    return _unique_positions(rng, W, H, count,
                             lambda g, m: (g.uniform(-0.5, W - 0.5, m), g.uniform(-0.5, H - 0.5, m)))


def tsv_clustered_xy(rng, W, H, count, n_clusters, sigma, taken_xy=None):
    """Isotropic Gaussian clusters, centres uniform, TSVs split evenly across clusters."""
    cx = rng.uniform(0, W - 1, n_clusters)
    cy = rng.uniform(0, H - 1, n_clusters)
    per = np.full(n_clusters, count // n_clusters)
    per[: count % n_clusters] += 1
    owner = np.repeat(np.arange(n_clusters), per)
    state = {"i": 0}

    def draw(g, m):
        idx = owner[(state["i"] + np.arange(m)) % count]
        state["i"] += m
        return g.normal(cx[idx], sigma), g.normal(cy[idx], sigma)

    return _unique_positions(rng, W, H, count, draw)


def _columns(T, xs, ys, r_each):
    """Through-stack TSV columns: one segment per adjacent tier pair, each with the TSV's R."""
    tsv = []
    for x, y, r in zip(xs, ys, r_each):
        for t in range(T - 1):
            tsv.append((t, int(x), int(y), float(r)))
    return tsv


def _pads_on_pitch(W, H, pitch, r, tier=0):
    return [(tier, x, y, r) for y in range(0, H, pitch) for x in range(0, W, pitch)]


# --------------------------------------------------------------------------
# the workloads
# --------------------------------------------------------------------------

def tiny_plain(seed=BASE_SEED + 0) -> Instance:
    """2 tiers x 32x32 (2,048 nodes): x/y segments 0.05 ohm (tier 0) and 0.10 ohm (tier 1),
    each x lognormal(0.1); 16 TSVs of 0.02 ohm at uniform distinct positions; pads of
    0.01 ohm on tier 0 on an 8-node pitch (16 pads)."""
    rng = np.random.default_rng(seed)
    T, W, H = 2, 32, 32
    base = [0.05, 0.10]
    rx = np.stack([_jittered(rng, base[t], (H, W - 1), 0.1) for t in range(T)])
    ry = np.stack([_jittered(rng, base[t], (H - 1, W), 0.1) for t in range(T)])
    xs, ys = tsv_uniform_xy(rng, W, H, 16)
    tsv = _columns(T, xs, ys, np.full(16, 0.02))
    pads = _pads_on_pitch(W, H, 8, 0.01)
    inst = from_resistances(rx, ry, tsv, pads, "tiny_plain_2x32x32")
    inst.meta.update(k=128, seed=seed)
    return inst


def precision_4x512(seed=BASE_SEED + 1, W=512, H=512, T=4, n_tsv=2000, n_clusters=40,
                    pad_pitch=16, pad_r=0.01) -> Instance:
    """4 tiers x 512x512 (1,048,576 nodes): per-tier anisotropic r_x, r_y log-uniform on
    [0.02, 0.2] ohm with lognormal(0.2) jitter; 2,000 through-stack TSVs of R uniform on
    [0.01, 0.05] ohm in 40 Gaussian clusters (sigma W/32); pads on tier 0 on a 16-node pitch."""
    rng = np.random.default_rng(seed)
    lo, hi = np.log(0.02), np.log(0.2)
    rx = np.empty((T, H, W - 1))
    ry = np.empty((T, H - 1, W))
    for t in range(T):
        r_x, r_y = np.exp(rng.uniform(lo, hi, 2))
        rx[t] = _jittered(rng, r_x, (H, W - 1), 0.2)
        ry[t] = _jittered(rng, r_y, (H - 1, W), 0.2)
    xs, ys = tsv_clustered_xy(rng, W, H, n_tsv, n_clusters, W / 32)
    r_t = rng.uniform(0.01, 0.05, n_tsv)
    tsv = _columns(T, xs, ys, r_t)
    pads = _pads_on_pitch(W, H, pad_pitch, pad_r)
    inst = from_resistances(rx, ry, tsv, pads, f"precision_{T}x{W}x{H}")
    inst.meta.update(k=256, seed=seed)
    return inst


def large_8x1024(seed=BASE_SEED + 2, W=1024, H=1024, T=8, n_tsv=20000, open_frac=0.10) -> Instance:
    """8 tiers x 1024x1024 (8,388,608 nodes): tiers alternate 0.1 ohm (even) and 0.02 ohm (odd),
    lognormal(0.2) jitter, 10% of segments open; 20,000 TSV columns (70% in 80 clusters, 30%
    uniform) of R uniform on [0.01, 0.05]; pads of 0.005 ohm on tier 0 on a 32-node pitch."""
    rng = np.random.default_rng(seed)
    rx = np.empty((T, H, W - 1))
    ry = np.empty((T, H - 1, W))
    for t in range(T):
        base = 0.1 if t % 2 == 0 else 0.02
        rx[t] = _jittered(rng, base, (H, W - 1), 0.2)
        ry[t] = _jittered(rng, base, (H - 1, W), 0.2)
    rx[rng.random(rx.shape) < open_frac] = np.inf
    ry[rng.random(ry.shape) < open_frac] = np.inf
    n_cl = int(round(0.7 * n_tsv))
    xs1, ys1 = tsv_clustered_xy(rng, W, H, n_cl, 80, W / 32)
    taken = set(zip(xs1.tolist(), ys1.tolist()))
    xs2, ys2 = [], []
    while len(xs2) < n_tsv - n_cl:
        x, y = (int(v) for v in rng.integers(0, [W, H]))
        if (x, y) not in taken:
            taken.add((x, y))
            xs2.append(x)
            ys2.append(y)
    xs = np.concatenate([xs1, np.array(xs2, dtype=np.int32)])
    ys = np.concatenate([ys1, np.array(ys2, dtype=np.int32)])
    r_t = rng.uniform(0.01, 0.05, n_tsv)
    tsv = _columns(T, xs, ys, r_t)
    pads = _pads_on_pitch(W, H, 32, 0.005)
    inst = from_resistances(rx, ry, tsv, pads, f"large_{T}x{W}x{H}")
    inst.meta.update(k=256, seed=seed)
    return inst


def batch_candidate(rng, idx=0, T=None, W=None, n_tsv=None, clustered=None) -> Instance:
    """One TSV-placement candidate: 2-4 tiers, W=H in {64,128,256}, 50-800 TSV columns placed
    uniformly or in clusters, the precision-workload resistance distributions, pads of 0.01 ohm
    on tier 0 on a 16-node pitch."""
    T = int(rng.integers(2, 5)) if T is None else T
    W = int(rng.choice([64, 128, 256])) if W is None else W
    H = W
    n_tsv = int(rng.integers(50, 801)) if n_tsv is None else n_tsv
    clustered = bool(rng.integers(0, 2)) if clustered is None else clustered
    lo, hi = np.log(0.02), np.log(0.2)
    rx = np.empty((T, H, W - 1))
    ry = np.empty((T, H - 1, W))
    for t in range(T):
        r_x, r_y = np.exp(rng.uniform(lo, hi, 2))
        rx[t] = _jittered(rng, r_x, (H, W - 1), 0.2)
        ry[t] = _jittered(rng, r_y, (H - 1, W), 0.2)
    if clustered:
        xs, ys = tsv_clustered_xy(rng, W, H, n_tsv, max(1, n_tsv // 50), W / 32)
    else:
        xs, ys = tsv_uniform_xy(rng, W, H, n_tsv)
    r_t = rng.uniform(0.01, 0.05, n_tsv)
    inst = from_resistances(rx, ry, _columns(T, xs, ys, r_t), _pads_on_pitch(W, H, 16, 0.01),
                            f"cand{idx}_{T}x{W}x{H}_{n_tsv}{'c' if clustered else 'u'}")
    inst.meta.update(k=64)
    return inst


def batch_candidates(count=512, seed=BASE_SEED + 3) -> list[Instance]:
    """The batching workload: `count` uneven TSV-placement candidates."""
    rng = np.random.default_rng(seed)
    return [batch_candidate(rng, i) for i in range(count)]


def random_small(rng, T=None, W=None, H=None, n_tsv=None, n_pads=None, open_frac=0.0,
                 sigma=0.5) -> Instance:
    """Small random instance for parity and property tests (ragged sizes allowed)."""
    T = int(rng.integers(1, 4)) if T is None else T
    W = int(rng.integers(1, 9)) if W is None else W
    H = int(rng.integers(1, 9)) if H is None else H
    base = rng.uniform(0.02, 0.2, T)
    rx = np.stack([_jittered(rng, base[t], (H, W - 1), sigma) for t in range(T)])
    ry = np.stack([_jittered(rng, base[t], (H - 1, W), sigma) for t in range(T)])
    if open_frac > 0:
        rx[rng.random(rx.shape) < open_frac] = np.inf
        ry[rng.random(ry.shape) < open_frac] = np.inf
    tsv = []
    if T > 1:
        n_tsv = int(rng.integers(1, 1 + max(1, W * H // 2))) if n_tsv is None else n_tsv
        for _ in range(n_tsv):
            tsv.append((int(rng.integers(0, T - 1)), int(rng.integers(0, W)),
                        int(rng.integers(0, H)), float(rng.uniform(0.01, 0.05))))
    n_pads = int(rng.integers(1, 4)) if n_pads is None else n_pads
    pads = [(0, int(rng.integers(0, W)), int(rng.integers(0, H)), float(rng.uniform(0.005, 0.02)))
            for _ in range(n_pads)]
    return from_resistances(rx, ry, tsv, pads, f"rand_{T}x{W}x{H}")


def precision_2x512(seed=BASE_SEED + 1) -> Instance:
    """Half of the precision recipe (2 tiers x 512 x 512, 1,000 TSV columns in 20 clusters):
    the small case on which profiler captures of the solver kernels run."""
    return precision_4x512(seed=seed, T=2, n_tsv=1000, n_clusters=20)


WORKLOADS = {
    "tiny_plain_2x32x32": tiny_plain,
    "precision_2x512x512": precision_2x512,
    "precision_4x512x512": precision_4x512,
    "large_8x1024x1024": large_8x1024,
}
