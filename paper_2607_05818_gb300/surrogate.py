"""Learned surrogate of the R map for TSV-planning sweeps (data, training, screening).

The network is the library's BF16 U-Net (er_surrogate_*): its forward and backward
kernels, loss and Adam all run in liber.so; this module only encodes networks as per-node
maps, produces labels with the exact solver (the batching form of the JL + PCG path), and
drives training and screening.  The solver stays the judge: screening re-checks the
candidates the surrogate ranks worst, plus a random sample, with er_batch_solve.

Maps (per tier t, channels 4t..4t+3): x-conductance of the segment to x+1 and
y-conductance of the segment to y+1, a TSV map (where a TSV segment meets the node) and a
pad map; zero-padded to 32 channels.  Each conductance g enters as ln(1 + g) / 4 (0 at the
mesh edge, for an open segment or where there is no TSV or pad), so that the network sees
the logarithm of what it must map to log R (R scales as 1/g) and all channels are O(1).
Targets: natural log of each node's R (JL estimate, FP64 path), masked where R is
infinite (floating nodes).
"""
from __future__ import annotations

import time

import numpy as np

from . import instances as I

def _enc(g):
    return np.log1p(np.asarray(g, dtype=np.float64)) / 4.0


def node_maps(inst, in_ch: int = 32) -> np.ndarray:
    """[H][W][in_ch] float32 per-node maps of one network."""
    T, W, H = inst.T, inst.W, inst.H
    if 4 * T > in_ch:
        raise ValueError("in_ch too small for the tier count")
    m = np.zeros((H, W, in_ch), dtype=np.float32)
    for t in range(T):
        m[:, : W - 1, 4 * t] = _enc(inst.gx[t])
        m[: H - 1, :, 4 * t + 1] = _enc(inst.gy[t])
    # parallel TSVs at one node add their conductances
    for tier, x, y, g in zip(inst.tsv_tier, inst.tsv_x, inst.tsv_y, inst.tsv_g):
        for t in (tier, tier + 1):
            cur = np.expm1(4.0 * m[y, x, 4 * t + 2])
            m[y, x, 4 * t + 2] = _enc(cur + g)
    for tier, x, y, g in zip(inst.pad_tier, inst.pad_x, inst.pad_y, inst.pad_g):
        cur = np.expm1(4.0 * m[y, x, 4 * tier + 3])
        m[y, x, 4 * tier + 3] = _enc(cur + g)
    return m


def target_map(R: np.ndarray, inst):
    """(log R [H][W][T] float32, mask uint8) from a node-ordered R vector."""
    r = R.reshape(inst.T, inst.H, inst.W).transpose(1, 2, 0)
    mask = np.isfinite(r)
    t = np.where(mask, np.log(np.where(mask, r, 1.0)), 0.0).astype(np.float32)
    return t, mask.astype(np.uint8)


def candidate(rng, T=4, W=256):
    """One TSV-placement candidate of the surrogate workload (random mesh resistances and TSV
    layout, as in the batching workload)."""
    return I.batch_candidate(rng, T=T, W=W)


def bf16_bits(a: np.ndarray) -> np.ndarray:
    """float32 -> BF16 bit patterns (uint16), round to nearest even (finite inputs)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    return ((u + (0x7FFF + ((u >> 16) & 1))) >> 16).astype(np.uint16)


def candidate_at(seed: int, i: int, T: int = 4, W: int = 256):
    """Candidate i of the seeded set `seed` (its own generator, so any subset can be rebuilt)."""
    return candidate(np.random.default_rng([seed, i]), T=T, W=W)


def _maps_worker(args):
    seed, lo, hi, T, W, in_ch = args
    return lo, np.stack([bf16_bits(node_maps(candidate_at(seed, i, T, W), in_ch)) for i in range(lo, hi)])


def upload_maps(count: int, seed: int, T: int = 4, W: int = 256, in_ch: int = 32, workers: int = 0, device="cuda"):
    """Maps of candidates 0..count-1 of the seeded set, encoded by `workers` spawned processes
    (0: this process) and copied chunk by chunk into one BF16 device tensor [count][W][W][in_ch]."""
    import torch
    out = torch.empty((count, W, W, in_ch), dtype=torch.bfloat16, device=device)
    chunks = [(seed, lo, min(count, lo + 32), T, W, in_ch) for lo in range(0, count, 32)]

    def put(lo, bits):
        out[lo:lo + bits.shape[0]].view(torch.int16).copy_(torch.from_numpy(bits.view(np.int16)))

    if workers > 0 and len(chunks) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(workers) as pool:
            for lo, bits in pool.imap_unordered(_maps_worker, chunks):
                put(lo, bits)
    else:
        for c in chunks:
            put(*_maps_worker(c))
    return out


def label(nets, k: int, seed: int, chunk: int = 64):
    """Exact-solver labels: R maps of `nets` with the batching form (network c uses seed + c)."""
    import torch

    from . import er
    out = []
    for lo in range(0, len(nets), chunk):
        part = nets[lo:lo + chunk]
        grids = [er.grid_create(n) for n in part]
        R = [torch.empty(n.n, dtype=torch.float64, device="cuda") for n in part]
        er.batch_solve(grids, k, seed + lo, R)
        torch.cuda.synchronize()
        out += [r.cpu().numpy() for r in R]
        for g in grids:
            g.destroy()
    return out


def label_set(count: int, seed: int, k: int, label_seed: int, T: int = 4, W: int = 256, chunk: int = 64,
              device="cuda"):
    """Solver labels (log R maps and masks, on the device) of candidates 0..count-1 of the seeded
    set, rebuilt and solved `chunk` at a time with the batching form.  Returns (tgt, msk,
    seconds spent in grid creation and solves)."""
    import torch

    from . import er
    tgt = torch.empty((count, W, W, T), dtype=torch.float32, device=device)
    msk = torch.empty((count, W, W, T), dtype=torch.uint8, device=device)
    solve_s = 0.0
    for lo in range(0, count, chunk):
        part = [candidate_at(seed, i, T, W) for i in range(lo, min(count, lo + chunk))]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grids = [er.grid_create(n) for n in part]
        R = [torch.empty(n.n, dtype=torch.float64, device=device) for n in part]
        er.batch_solve(grids, k, label_seed + lo, R)
        torch.cuda.synchronize()
        solve_s += time.perf_counter() - t0
        for j, (n, r) in enumerate(zip(part, R)):
            t, m = target_map(r.cpu().numpy(), n)
            tgt[lo + j].copy_(torch.from_numpy(t))
            msk[lo + j].copy_(torch.from_numpy(m))
        for g in grids:
            g.destroy()
    return tgt, msk, solve_s


def to_device(nets, Rs, in_ch=32):
    """Stack maps (BF16), targets (FP32) and masks (uint8) on the GPU."""
    import torch
    maps = torch.from_numpy(np.stack([node_maps(n, in_ch) for n in nets])).to("cuda", torch.bfloat16)
    tm = [target_map(R, n) for R, n in zip(Rs, nets)]
    tgt = torch.from_numpy(np.stack([t for t, _ in tm])).cuda()
    msk = torch.from_numpy(np.stack([m for _, m in tm])).cuda()
    return maps, tgt, msk


def train(model, maps, tgt, msk, epochs: int, batch: int, lr: float, seed: int = 0, log=None,
          lr_final: float | None = None):
    """Adam on the masked MSE of log R; returns the per-epoch mean loss.  The step size
    falls from lr to lr_final (default: lr) along a cosine over the epochs.  Before the first
    step the head's biases are set to the per-tier mean of the masked targets, so that the
    network starts from the mean map's level instead of 0."""
    rng = np.random.default_rng(seed)
    n = maps.shape[0]
    if model.step_count() == 0:
        m = msk.float()
        mean = ((tgt * m).sum(dim=(0, 1, 2)) / m.sum(dim=(0, 1, 2)).clamp(min=1)).cpu().numpy()
        p = model.get_params()
        p[-len(mean):] = mean
        model.set_params(p)
    hist = []
    lr_final = lr if lr_final is None else lr_final
    for ep in range(epochs):
        lr_ep = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * ep / max(epochs - 1, 1)))
        order = rng.permutation(n)
        tot, cnt = 0.0, 0
        for lo in range(0, n - batch + 1, batch):
            idx = order[lo:lo + batch]
            tot += model.train_step(maps[idx].contiguous(), tgt[idx].contiguous(), msk[idx].contiguous(), batch, lr_ep)
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep}: loss {hist[-1]:.4f}")
    return hist


def predict(model, maps, batch: int):
    import torch
    n = maps.shape[0]
    out = torch.empty((n,) + tuple(maps.shape[1:3]) + (model.shape.out_ch,), dtype=torch.float32, device="cuda")
    for lo in range(0, n, batch):
        b = min(batch, n - lo)
        model.infer(maps[lo:lo + b].contiguous(), b, out[lo:lo + b])
    torch.cuda.synchronize()
    return out


def score(logR, mask=None):
    """Screening score of one candidate: the 99th percentile of log R over its (finite) nodes,
    the level of its worst nodes without the JL noise of a single node."""
    v = np.asarray(logR).ravel()
    if mask is not None:
        v = v[np.asarray(mask).ravel().astype(bool)]
    return float(np.percentile(v, 99)) if v.size else -np.inf


def rel_errors(pred_logR, R_exact, inst):
    """Per-node relative error of exp(predicted log R) against R (finite nodes only)."""
    t, m = target_map(R_exact, inst)
    p = np.exp(pred_logR)
    r = np.exp(t)
    e = np.abs(p / r - 1.0)[m.astype(bool)]
    return e


def screen(model, cands, k: int, seed: int, frac: float = 0.05, batch: int = 8):
    """Surrogate-then-verify sweep: rank candidates by the surrogate's worst (largest) R, re-check
    the worst `frac` and a random `frac` with the exact solver, report the surrogate's errors on
    them and the times of both stages."""
    import torch
    t0 = time.perf_counter()
    maps = torch.from_numpy(np.stack([node_maps(c) for c in cands])).to("cuda", torch.bfloat16)
    t1 = time.perf_counter()
    pred = predict(model, maps, batch).cpu().numpy()
    t2 = time.perf_counter()
    sc = np.array([score(p) for p in pred])
    nv = max(1, int(round(frac * len(cands))))
    worst = np.argsort(-sc)[:nv]
    rng = np.random.default_rng(seed)
    rand = rng.choice(np.setdiff1d(np.arange(len(cands)), worst), size=min(nv, len(cands) - nv), replace=False)
    check = np.concatenate([worst, rand])
    t3 = time.perf_counter()
    Rs = label([cands[i] for i in check], k, seed)
    t4 = time.perf_counter()
    errs = [rel_errors(pred[i], R, cands[i]) for i, R in zip(check, Rs)]
    allerr = np.concatenate(errs)
    return {"candidates": len(cands), "verified": len(check), "surrogate_s": (t2 - t1), "encode_s": t1 - t0,
            "verify_s": t4 - t3, "max_rel_err": float(allerr.max()), "mean_rel_err": float(allerr.mean()),
            "worst_max_rel_err": float(np.concatenate(errs[:nv]).max()),
            "random_mean_rel_err": float(np.concatenate(errs[nv:]).mean()) if len(rand) else None}
