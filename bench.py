"""Benchmark: all-node effective-resistance map throughput (nodes/s) on one GB300 per rank.

One step = the whole hot path on one synthetic network already resident in HBM:
JL sketch (er_sketch) + k-RHS preconditioned CG solve (er_solve; multigrid V-cycle by
default) + R map (er_reff_map).
Default workload: 4 tiers x 512x512 (1,048,576 nodes), k = 256, the FP32 form: FP32
vectors and stencil, double-float dot sums, a double-float iterate (pairs of FP32 numbers)
with the accurate residual substituted every 50 iterations (reliable updates), stopped at an
accurate residual of 1e-7, with the aggregation-multigrid V-cycle as preconditioner
(--precond jacobi: Jacobi-PCG).

Prints one JSON line (rank 0).  N > 1 (torchrun): every rank maps its own network
(independent seeds) with no collective on the data path; value = all ranks' nodes /
the slowest rank's time (weak scaling).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--prec fp32|fp64] [--no-accuracy]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "R_eff map nodes/s at <=1e-3 max rel err (FP32+refinement vs plain FP64)"
UNIT = "nodes/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="precision_4x512x512")
    p.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    p.add_argument("--precond", default="mg", choices=["jacobi", "mg"],
                   help="FP32 form: Jacobi or aggregation-multigrid V-cycle preconditioner")
    p.add_argument("--k", type=int, default=256)
    p.add_argument("--shard", default="replicas", choices=["replicas", "columns"],
                   help="N > 1: every rank maps its own network (replicas, weak scaling), or all ranks map "
                        "one network, each solving its share of the sketch columns, and the partial maps are "
                        "summed (columns, strong scaling)")
    p.add_argument("--tol", type=float, default=None)
    p.add_argument("--no-accuracy", action="store_true")
    p.add_argument("--acc-block", type=int, default=0,
                   help="solve the plain FP64 reference in blocks of this many sketch columns (0: all at once)")
    p.add_argument("--cpu-sample", type=int, default=256, help="W=H of the oracle's bounded sample")
    p.add_argument("--batch-count", type=int, default=512, help="candidates of the batching workload")
    p.add_argument("--no-autotune", action="store_true",
                   help="batching workload: library default tile rows instead of the autotuner's per size class")
    p.add_argument("--sur-train", type=int, default=1024, help="surrogate workload: solver-labelled training configs")
    p.add_argument("--sur-screen", type=int, default=4096, help="surrogate workload: screened candidates")
    p.add_argument("--sur-k", type=int, default=64, help="surrogate workload: JL columns of labels and verification")
    p.add_argument("--sur-epochs", type=int, default=12)
    p.add_argument("--sur-batch", type=int, default=128, help="surrogate workloads: candidates per forward call")
    p.add_argument("--sur-recall", type=int, default=512, help="surrogate workload: candidates solved exactly "
                                                                "to measure the screen's recall (untimed)")
    p.add_argument("--workers", type=int, default=8, help="spawned processes encoding candidate maps")
    return p.parse_args()


def make_workload(name, rank=0):
    from paper_2607_05818_gb300 import instances as I
    if name not in I.WORKLOADS:
        raise SystemExit(f"unknown workload {name}; choose from {sorted(I.WORKLOADS)}")
    fn = I.WORKLOADS[name]
    inst = fn() if rank == 0 else fn(seed=I.BASE_SEED + 1000 + rank)
    return inst


def cpu_sample_instance(W):
    """The bounded sample the oracle is timed on: the 4-tier precision recipe at W x W with
    TSV and cluster counts scaled by area."""
    from paper_2607_05818_gb300 import instances as I
    f = (W / 512) ** 2
    return I.precision_4x512(W=W, H=W, n_tsv=max(1, int(round(2000 * f))), n_clusters=max(1, int(round(40 * f))))


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the CPU-baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_step(inst, k, seed, threads=None):
    """The CPU oracle as it stands, phase by phase: assembly and sparse LU factorisation of G
    (SuperLU, one thread), the C sketch, the k right-hand-side solves in column blocks of 8 on
    `threads` host threads, and the row norms.  Returns (seconds per phase, non-floating nodes,
    threads used)."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import exact
    from oracle import sketch as osk
    threads = threads or os.cpu_count() or 1
    ph = {}
    t0 = time.perf_counter()
    f = exact.SparseFactor(inst)
    ph["factor_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    Yt = osk.sketch(inst, k, seed)
    ph["sketch_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    blocks = list(range(0, k, 8))
    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(lambda j: f.solve(Yt[:, j:j + 8]), blocks))
    ph["solves_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    R = sum(np.sum(Z * Z, axis=1) for Z in parts)
    R[f.floating] = np.inf
    ph["row_norms_s"] = time.perf_counter() - t0
    ph["total_s"] = sum(ph.values())
    return ph, int(np.sum(~f.floating)), threads


def cpu_baseline(args):
    """The oracle timed on the host cores on two bounded samples of the bench recipe (4 tiers of
    128^2 and 256^2), phases separately; the 4 x 512^2 figure is extrapolated from the measured
    growth of each phase between the two samples (labelled as such)."""
    from oracle import build as ob
    ob.build()
    res = {}
    for W in (args.cpu_sample // 2, args.cpu_sample):
        inst = cpu_sample_instance(W)
        ph, n_ok, thr = oracle_step(inst, args.k, inst.meta.get("seed", 1))
        res[W] = (ph, n_ok, inst)
    (ph_s, n_s, _), (ph_l, n_l, inst_l) = res[args.cpu_sample // 2], res[args.cpu_sample]
    n_bench = 4 * 512 * 512
    est = 0.0
    growth = {}
    for key in ("factor_s", "sketch_s", "solves_s", "row_norms_s"):
        a = np.log(max(ph_l[key], 1e-9) / max(ph_s[key], 1e-9)) / np.log(n_l / n_s)
        growth[key] = float(a)
        est += ph_l[key] * (n_bench / n_l) ** max(a, 1.0)
    return {"value": n_l / ph_l["total_s"], "unit": UNIT, "cores": thr, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "sample": f"one {inst_l.T}x{inst_l.W}x{inst_l.H} network ({inst_l.n} nodes) of the bench recipe, k={args.k}: "
                      f"SuperLU factorisation (1 thread), C sketch, {args.k} sparse solves in blocks of 8 on {thr} "
                      f"threads, row norms",
            "phases_s": {k_: round(v, 3) for k_, v in ph_l.items()},
            "phases_s_smaller_sample": {k_: round(v, 3) for k_, v in ph_s.items()},
            "same_config": False,
            "extrapolated_bench_network": {
                "value": n_bench / est, "unit": UNIT, "seconds": est,
                "note": "4x512x512: each phase scaled from the 256^2 sample by its measured growth exponent "
                        "between the 128^2 and 256^2 samples (at least linear)", "growth_exponents": growth}}


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower() == "active"})
        pw = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "power_w_max": max(pw) if pw else None}


def combine_ranks(units, seconds, world, device="cpu"):
    """Whole-job figures over the ranks: (sum of the units every rank processed, the slowest
    rank's time).  Each rank works on its own independent problems, so this is the only
    exchange, and it happens after the timed region."""
    if world <= 1:
        return float(units), float(seconds)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    n = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n)
    return float(n.item()), float(t.item())


def reduce_partial_map(R, world):
    """Column sharding: R_i = sum_j Z_ij^2 runs over independent sketch columns, so the map of the
    whole sketch is the sum of the ranks' partial maps over their column shards.  One sum
    all-reduce of the n-vector (in place; NCCL on GPUs, gloo on CPU) is the only exchange."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(R, op=dist.ReduceOp.SUM)
    return R


def load_peaks():
    """Measured HBM and BF16 peaks of this GPU model, else the stated fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        parts = [p for p in vis.split(",") if p.strip()]
        if local_rank < len(parts):
            return parts[local_rank].strip()
    return str(local_rank)


def kernel_source_hash():
    """Hash of the solver kernels' device code: the multigrid kernels (er_mg.cu up to its host
    section), the FP32 and FP64 passes and their shared device helpers.  A change there makes
    the committed DRAM counters stale."""
    h = hashlib.sha256()
    for f in ("er_pcg.cu", "er_fp32.cu", "er_mg.cu", "er_common.cuh"):
        text = open(os.path.join(ROOT, "paper_2607_05818_gb300", "csrc", f), "rb").read()
        if f == "er_mg.cu":
            text = text.split(b"// ---- tensor maps of the tiled kernels")[0]
        h.update(text)
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or None when the
    kernel source has changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        d = json.load(open(path))
    except (OSError, ValueError):
        return None
    e = d.get(kernel, {})
    if e.get("source_hash") != kernel_source_hash() or e.get("workload") != workload:
        return None
    return e.get("dram_bytes_per_launch")


def run_batch(args, rank, world, local_rank):
    """Batching form: 512 TSV-placement candidates (k = 64) through er_batch_solve, with the
    multigrid preconditioner (every pass one persistent launch over all running networks, the
    loop a device-side graph node; the default, --precond mg) or Jacobi (shared launches), the
    other mode timed once beside it, against the same candidates solved one after another
    (er_solve per candidate, warm workspace)."""
    import torch
    from paper_2607_05818_gb300 import er
    from paper_2607_05818_gb300 import instances as I

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    k = 64
    cands = I.batch_candidates(args.batch_count, seed=I.BASE_SEED + 3 + 1000 * rank)
    grids = [er.grid_create(c) for c in cands]
    infos = [g.info() for g in grids]
    n_ok = sum(i["n_nodes"] - i["n_floating"] for i in infos)
    R = [torch.empty(c.n, dtype=torch.float64, device=dev) for c in cands]
    opts = er.default_solve_opts("fp32")
    opts_mg = er.default_solve_opts("fp32", precond=1, check_every=2)
    if args.tol is not None:
        opts.tol = args.tol
        opts_mg.tol = args.tol
    use_mg = args.precond == "mg"
    opts_run, opts_other = (opts_mg, opts) if use_mg else (opts, opts_mg)
    rows = None
    t_tune = 0.0
    if not args.no_autotune:  # per size class (tiers, W, H), measured once, outside the timed region
        from paper_2607_05818_gb300 import autotune
        tt = time.perf_counter()
        rows = [autotune.best_mg_order(c, k) if use_mg else autotune.best_rows(c, k) for c in cands]
        t_tune = time.perf_counter() - tt
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        er.batch_solve(grids, k, 1, R, opts=opts_run, tile_rows=rows)
    torch.cuda.synchronize()
    stats = []
    with ClockSampler(gpu_index(local_rank)) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(er.batch_solve(grids, k, 1, R, opts=opts_run, tile_rows=rows)[1])
        e1.record(stream)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
    n_job, s_max = combine_ranks(n_ok, e0.elapsed_time(e1) / 1e3, world, dev)
    ms = 1e3 * s_max
    value = n_job * args.steps / s_max
    # the other mode of er_batch_solve, one call (outside the timed region)
    o0 = time.perf_counter()
    st_other = er.batch_solve(grids, k, 1, R, opts=opts_other)[1]  # library default launch shape
    torch.cuda.synchronize()
    other_s = time.perf_counter() - o0
    # sequential: each candidate's sketch + solve + map on its own (second call, warm workspace),
    # with the batching form's Jacobi preconditioner and with the multigrid V-cycle
    nmax = max(c.n for c in cands)
    Y = torch.empty(nmax * k, dtype=torch.float32, device=dev)
    Z = torch.empty_like(Y)
    seq_ms, seq_mg_ms = 0.0, 0.0
    for c, (cand, g) in enumerate(zip(cands, grids)):
        y = Y[: cand.n * k].view(cand.n, k)
        z = Z[: cand.n * k].view(cand.n, k)
        for o, which in ((opts, 0), (opts_mg, 1)):
            for rep in range(2):
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                er.sketch(g, k, 1 + c, "fp32", y)
                er.solve(g, y, z, k, "fp32", o)
                er.reff_map(g, z, k, "fp32", R[c])
                a1.record(stream)
                torch.cuda.synchronize()
                if rep == 1:
                    if which == 0:
                        seq_ms += a0.elapsed_time(a1)
                    else:
                        seq_mg_ms += a0.elapsed_time(a1)
        g.destroy()
    seq_value = n_ok / (seq_ms / 1e3)
    seq_mg_value = n_ok / (seq_mg_ms / 1e3)
    last = stats[-1]
    return {
        "metric": "batched R_eff map nodes/s (512 TSV-placement candidates, FP32 form)", "value": value,
        "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"batch_candidates_{len(cands)}", "k": k, "candidates": len(cands),
                   "nodes": n_ok, "iterations": last["iterations"], "converged": last["converged"],
                   "graph_captures": last["graph_captures"],
                   "launch_shape": (f"autotuned per size class ({'launch order' if use_mg else 'tile rows'}: "
                                    f"{sorted(set(rows))}, {t_tune:.1f} s to tune, untimed)" if rows
                                    else "library default"),
                   "max_rel_residual": last["max_rel_residual"],
                   "mode": "multigrid: every pass one persistent launch over the running networks, loop in a device-side graph node"
                   if use_mg else "Jacobi: shared launches over a (network, tile) work list"},
        "other_mode": {"mode": "Jacobi shared launches" if use_mg else "multigrid graph of all networks",
                       "value": n_ok / other_s, "unit": UNIT, "seconds": other_s,
                       "iterations": st_other["iterations"], "converged": st_other["converged"],
                       "note": "one er_batch_solve call, host wall time"},
        "sequential": {"value": seq_value, "unit": UNIT, "ms": seq_ms,
                       "note": "er_sketch + er_solve + er_reff_map per candidate, warm workspace, Jacobi"},
        "sequential_multigrid": {"value": seq_mg_value, "unit": UNIT, "ms": seq_mg_ms,
                                 "note": "as sequential, with the multigrid preconditioner"},
        "batched_over_sequential": value / seq_value,
        "gpu_launches": int(sum(s["launches"] for s in stats)), "clocks": clk.summary(),
    }


def unet_conv_flops(levels, base, in_ch, H, W):
    """Multiply-add flops (x2) of the U-Net's 3x3 convolutions for one sample."""
    f = 0
    for l in range(levels):
        c, hw = base << l, (H >> l) * (W >> l)
        f += 2 * hw * 9 * c * ((in_ch if l == 0 else base << (l - 1)) + c)
    for l in range(levels - 2, -1, -1):
        c, hw = base << l, (H >> l) * (W >> l)
        f += 2 * hw * 9 * c * ((base << (l + 1)) + 2 * c)
    return f


def run_surrogate(args, rank, world, local_rank):
    """Learned-surrogate form on 4-tier 256x256 candidates: a 6-level, 32-base-channel BF16
    U-Net trained (untimed setup) on solver labels of seeded random TSV layouts; one step
    screens the candidate set with the surrogate, then re-solves the worst 5% and a random 5%
    with the exact path (batching form), whose maps are the ones returned for them."""
    import torch
    from paper_2607_05818_gb300 import er
    from paper_2607_05818_gb300 import surrogate as S

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    T, W, L, C, in_ch = 4, 256, 6, 32, 32
    n_nodes = T * W * W
    seed_tr, seed_sc = 70001 + 1000 * rank, 80001 + 1000 * rank
    k = args.sur_k
    t0 = time.perf_counter()
    maps_tr = S.upload_maps(args.sur_train, seed_tr, T, W, in_ch, workers=args.workers, device=dev)
    maps_sc = S.upload_maps(args.sur_screen, seed_sc, T, W, in_ch, workers=args.workers, device=dev)
    t_maps = time.perf_counter() - t0
    tgt, msk, t_label = S.label_set(args.sur_train, seed_tr, k, 1, T, W, device=dev)
    model = er.Surrogate(in_ch=in_ch, out_ch=T, levels=L, base=C, H=W, W=W, seed=3)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = S.train(model, maps_tr, tgt, msk, epochs=args.sur_epochs, batch=8, lr=1e-3, lr_final=1e-4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    del tgt, msk, maps_tr
    nb = args.sur_batch  # candidates per forward call: enough pixel tiles to fill the SMs at the deep levels
    pred = torch.empty((args.sur_screen, W, W, T), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    fwd_launches = 6 * L - 3  # 2L convolutions, L-1 pools, L-1 upsamplings, 2(L-1) decoder convolutions, head

    def step(verify=True):
        """(forward ms by events, forward+rank s, verify s, flagged ids, verified R, stats)."""
        torch.cuda.synchronize()
        ta = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for lo in range(0, args.sur_screen, nb):
            b = min(nb, args.sur_screen - lo)
            model.infer(maps_sc[lo:lo + b], b, pred[lo:lo + b])
        e1.record(stream)
        score = np.concatenate([pred[lo:lo + 256].amax(dim=(1, 2, 3)).cpu().numpy()
                                for lo in range(0, args.sur_screen, 256)])
        torch.cuda.synchronize()
        fwd_s = time.perf_counter() - ta
        nv = max(1, int(round(0.05 * args.sur_screen)))
        worst = np.argsort(-score)[:nv]
        rest = np.setdiff1d(np.arange(args.sur_screen), worst)
        rand = np.random.default_rng(5).choice(rest, size=min(nv, rest.size), replace=False)
        flagged = np.concatenate([worst, rand])
        if not verify:
            return e0.elapsed_time(e1), fwd_s, 0.0, flagged, None, None
        insts = [S.candidate_at(seed_sc, int(i), T, W) for i in flagged]  # the candidates' descriptions
        torch.cuda.synchronize()
        tb = time.perf_counter()
        Rv, stats = [], None
        for lo in range(0, len(insts), 64):
            part = insts[lo:lo + 64]
            grids = [er.grid_create(n) for n in part]
            R = [torch.empty(n.n, dtype=torch.float64, device=dev) for n in part]
            _, st = er.batch_solve(grids, k, 1 + lo, R)
            Rv += [r.cpu().numpy() for r in R]
            for g in grids:
                g.destroy()
            stats = st if stats is None else {kk: stats[kk] + st[kk] if isinstance(st[kk], (int, float)) else st[kk]
                                             for kk in st}
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), fwd_s, time.perf_counter() - tb, flagged, (insts, Rv), stats

    for _ in range(args.warmup):
        step(verify=False)
    step(verify=True) if args.steps > 0 else None
    recs = []
    with ClockSampler(gpu_index(local_rank)) as clk:
        if world > 1:
            torch.distributed.barrier()
        for _ in range(args.steps):
            recs.append(step())
        if world > 1:
            torch.distributed.barrier()
    fwd_ms = statistics.median(r[0] for r in recs)
    fwd_s = statistics.median(r[1] for r in recs)
    ver_s = statistics.median(r[2] for r in recs)
    flagged, (insts, Rv), stats = recs[-1][3], recs[-1][4], recs[-1][5]
    step_s = fwd_s + ver_s
    n_job, s_max = combine_ranks(args.sur_screen * n_nodes, step_s, world, dev)
    value = n_job / s_max
    exact = len(insts) * n_nodes / ver_s
    nv = len(flagged) // 2
    pn = pred.index_select(0, torch.as_tensor(flagged, device=dev)).cpu().numpy()
    errs = [S.rel_errors(pn[j], Rv[j], insts[j]) for j in range(len(flagged))]
    allerr = np.concatenate(errs)
    # screening recall on a bounded sample (untimed): the first n_rec candidates solved exactly,
    # ranked by the same statistic as the screen (largest log R); how many of the truly worst
    # 5% the surrogate's worst 5% (and 10%) contain
    n_rec = min(args.sur_recall, args.sur_screen)
    t_rec = time.perf_counter()
    true_score = []
    for lo in range(0, n_rec, 64):
        part = [S.candidate_at(seed_sc, i, T, W) for i in range(lo, min(lo + 64, n_rec))]
        grids = [er.grid_create(n) for n in part]
        Rr = [torch.empty(n.n, dtype=torch.float64, device=dev) for n in part]
        er.batch_solve(grids, k, 1 + lo, Rr)
        for r_ in Rr:
            r_ = r_.cpu().numpy()
            true_score.append(float(np.log(r_[np.isfinite(r_)].max())))
        for g_ in grids:
            g_.destroy()
    true_score = np.array(true_score)
    pred_score = pred[:n_rec].amax(dim=(1, 2, 3)).cpu().numpy()
    q = max(1, int(round(0.05 * n_rec)))
    worst = set(np.argsort(-true_score)[:q].tolist())
    order = np.argsort(-pred_score)
    recall = {"sample": f"the first {n_rec} screened candidates, solved exactly (k={k}), {time.perf_counter() - t_rec:.1f} s",
              "worst_5pct": q, "in_surrogate_worst_5pct": len(worst & set(order[:q].tolist())) / q,
              "in_surrogate_worst_10pct": len(worst & set(order[:2 * q].tolist())) / q,
              "rank_correlation": float(np.corrcoef(np.argsort(np.argsort(true_score)),
                                                    np.argsort(np.argsort(pred_score)))[0, 1])}
    flops = unet_conv_flops(L, C, in_ch, W, W) * args.sur_screen
    ach = flops / (fwd_ms / 1e3) / 1e12
    pk = load_peaks()
    peak = pk.get("bf16_tflops")
    launches = fwd_launches * ((args.sur_screen + nb - 1) // nb) + int(stats["launches"] if stats else 0)
    return {
        "metric": "surrogate-then-verify R_eff map nodes/s (worst 5% + random 5% re-solved exactly)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * step_s, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 (surrogate) + f32/f64 (verification)", "data": "synthetic",
        "config": {"workload": f"surrogate_{T}x{W}x{W}", "candidates": args.sur_screen, "verified": int(len(flagged)),
                   "unet": {"levels": L, "base": C, "in_ch": in_ch, "params": model.num_params()},
                   "train_configs": args.sur_train, "label_k": k, "epochs": args.sur_epochs,
                   "l2": "inputs larger than L2 (17 GB of maps)"},
        "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                     "frac": ach / peak if peak else None, "traffic": None,
                     "kernel": "whole U-Net forward (3x3 conv flops / forward time; pool and head included)",
                     "peak_source": pk["source"] + " bf16_tflops (burst)"},
        "exact": {"value": exact, "unit": UNIT, "note": "verification throughput: er_grid_create + er_batch_solve "
                                                       "(k=%d, FP32 form) on the flagged candidates" % k},
        "gain_over_exact": value / exact,
        "surrogate_only": {"value": args.sur_screen * n_nodes / fwd_s, "unit": UNIT,
                           "forward_ms_per_candidate": fwd_ms / args.sur_screen},
        "screening_recall": recall,
        "surrogate_error_vs_solver": {
            "max_rel_err": float(allerr.max()), "mean_rel_err": float(allerr.mean()),
            "flagged_mean_rel_err": float(np.concatenate(errs[:nv]).mean()),
            "random_mean_rel_err": float(np.concatenate(errs[nv:]).mean())},
        "setup": {"maps_s": t_maps, "label_solve_s": t_label, "train_s": t_train,
                  "train_loss_first_last": [hist[0], hist[-1]]},
        "gpu_launches": launches, "clocks": clk.summary(),
    }


def fp32_alu_peak(sm_mhz=None):
    """FP32 CUDA-core peak of the GB300: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x SM clock
    (the measured median under load when given, else the 2,070 MHz maximum)."""
    mhz = sm_mhz or 2070.0
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


def run_pairs(args, rank, world, local_rank):
    """Bump-to-load pair resistances and an IR-drop map from one solved sketch of the 4x512x512
    network (FP32 form, k = 256): the 1,024 pads as bumps x 10,000 seeded load nodes on the top
    tier (the paper's bump-load setting), and the drop of every node under 4 load-current
    scenarios drawn at the same loads.  Setup (sketch + solve) is untimed; one step is
    er_pair_reff + er_ir_drop."""
    import torch
    from paper_2607_05818_gb300 import er
    from paper_2607_05818_gb300 import instances as I

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    inst = I.precision_4x512(seed=I.BASE_SEED + 1 + 1000 * rank)
    k, seed, n_loads, S = args.k, int(inst.meta.get("seed", 1)), 10000, 4
    g = er.grid_create(inst)
    Yt = torch.empty((inst.n, k), dtype=torch.float32, device=dev)
    Z = torch.empty_like(Yt)
    er.sketch(g, k, seed, "fp32", Yt)
    er.solve(g, Yt, Z, k, "fp32")
    del Yt
    bumps = (inst.pad_tier.astype(np.int64) * inst.H + inst.pad_y) * inst.W + inst.pad_x
    rng = np.random.default_rng(5 + rank)
    top = (inst.T - 1) * inst.W * inst.H
    loads = top + rng.choice(inst.W * inst.H, n_loads, replace=False)
    cur = rng.uniform(0.0, 1e-3, (n_loads, S))
    Rp = torch.empty((len(bumps), n_loads), dtype=torch.float64, device=dev)
    D = torch.empty((inst.n, S), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step():
        a0, a1, a2 = ev(), ev(), ev()
        a0.record(stream)
        er.pair_reff(g, Z, k, "fp32", bumps, loads, Rp)
        a1.record(stream)
        er.ir_drop(g, Z, k, "fp32", loads, cur, D)
        a2.record(stream)
        return a0, a1, a2

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = []
    with ClockSampler(gpu_index(local_rank)) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record(stream)
        for _ in range(args.steps):
            evs.append(step())
        e1.record(stream)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
    npairs = len(bumps) * n_loads
    n_job, s_max = combine_ranks(npairs, e0.elapsed_time(e1) / 1e3, world, dev)
    value = n_job * args.steps / s_max
    pair_ms = statistics.median(a.elapsed_time(b) for a, b, _ in evs)
    drop_ms = statistics.median(b.elapsed_time(c) for _, b, c in evs)
    cs = clk.summary()
    peak_alu = fp32_alu_peak(cs.get("sm_mhz") if isinstance(cs, dict) else None)
    pair_flops = 3.0 * npairs * k  # per column: one subtraction and one FMA (2 flops)
    drop_bytes = inst.n * k * 4 + n_loads * k * 4 + inst.n * S * 8
    peaks = load_peaks()
    # the oracle's definitions on a bounded sample: 64 bumps x 10,000 loads and the drop of
    # all nodes of a 1/8 slice, on a seeded random Z of the same row length
    cpu = None
    if rank == 0 and world == 1:
        rs = np.random.default_rng(9)
        Zs = rs.standard_normal((inst.n // 8, k)) * 0.05
        fl = np.zeros(len(Zs), dtype=bool)
        lo = rs.choice(len(Zs), n_loads, replace=False)
        from oracle import pairs as op
        t0 = time.perf_counter()
        op.pair_reff_jl(Zs, fl, lo[:64], lo)
        t1 = time.perf_counter()
        op.ir_drop_jl(Zs, fl, lo, cur)
        t2 = time.perf_counter()
        cpu = {"value": 64 * n_loads / (t1 - t0), "unit": "pairs/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle.pairs.pair_reff_jl on 64 x {n_loads} pairs ({t1 - t0:.2f} s) and ir_drop_jl "
                         f"of {len(Zs)} nodes x {S} scenarios ({t2 - t1:.2f} s, "
                         f"{len(Zs) / (t2 - t1):.3g} nodes/s), random Z with k = {k}"}
    return {
        "metric": "bump-load pair effective resistances per second from the solved sketch (FP32 Z)",
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * s_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (differences) + f64 (sums)", "data": "synthetic",
        "config": {"workload": "pairs_4x512x512", "k": k, "bumps": int(len(bumps)), "loads": n_loads,
                   "drop_scenarios": S, "nodes": inst.n,
                   "l2": "Z is 1 GiB, larger than L2; the pair kernel re-reads its 11 MB of rows from L2"},
        "roofline": {"kernel": "k_pair_reff<float>", "bound": "alu", "achieved": pair_flops / (pair_ms / 1e3) / 1e12,
                     "peak": peak_alu, "unit": "TFLOP/s", "frac": pair_flops / (pair_ms / 1e3) / 1e12 / peak_alu,
                     "traffic": None, "avg_launch_ms": pair_ms, "flops_per_launch": pair_flops,
                     "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flops x median SM clock"},
        "roofline_other": [{"kernel": "er_ir_drop (k_drop_partial + k_drop_fold + k_drop_apply)", "bound": "hbm",
                            "achieved": drop_bytes / (drop_ms / 1e3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                            "frac": drop_bytes / (drop_ms / 1e3) / 1e9 / peaks["hbm_gbs"], "traffic": None,
                            "avg_call_ms": drop_ms, "algorithmic_bytes_per_call": drop_bytes,
                            "peak_source": peaks["source"] + " hbm_gbs"}],
        "ir_drop": {"value": inst.n / (drop_ms / 1e3), "unit": "nodes/s", "scenarios": S},
        "cpu_baseline": cpu,
        "gpu_launches": 4 * args.steps, "clocks": cs,
    }


def run_unet_forward(args, rank, world, local_rank):
    """The surrogate's forward alone: the 6-level, 32-base-channel BF16 U-Net (random He
    weights; the arithmetic does not depend on them) over --sur-screen random 4x256x256
    candidate maps in batches of --sur-batch (128), timed with CUDA events.  Isolates the tcgen05 convolution
    kernels from training and verification."""
    import torch
    from paper_2607_05818_gb300 import er

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    T, W, L, C, in_ch, nb = 4, 256, 6, 32, 32, args.sur_batch
    model = er.Surrogate(in_ch=in_ch, out_ch=T, levels=L, base=C, H=W, W=W, seed=3 + rank)
    gen = torch.Generator(device=dev)
    gen.manual_seed(11 + rank)
    maps = torch.rand((args.sur_screen, W, W, in_ch), generator=gen, device=dev).to(torch.bfloat16)
    out = torch.empty((args.sur_screen, W, W, T), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        for lo in range(0, args.sur_screen, nb):
            b = min(nb, args.sur_screen - lo)
            model.infer(maps[lo:lo + b], b, out[lo:lo + b])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    with ClockSampler(gpu_index(local_rank)) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
    n_job, s_max = combine_ranks(args.sur_screen * T * W * W, e0.elapsed_time(e1) / 1e3, world, dev)
    value = n_job * args.steps / s_max
    flops = unet_conv_flops(L, C, in_ch, W, W) * args.sur_screen * args.steps
    ach = flops / (e0.elapsed_time(e1) / 1e3) / 1e12
    pk = load_peaks()
    return {
        "metric": "surrogate forward R_eff-map nodes/s (BF16 U-Net on tcgen05)", "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * s_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)",
        "data": "synthetic",
        "config": {"workload": "unet_forward_4x256x256", "candidates": args.sur_screen, "batch": nb,
                   "unet": {"levels": L, "base": C, "in_ch": in_ch, "params": model.num_params()},
                   "l2": f"inputs larger than L2 ({args.sur_screen * W * W * in_ch * 2 / 1e9:.1f} GB of maps)"},
        "roofline": {"bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                     "frac": ach / pk["bf16_tflops"], "traffic": None,
                     "kernel": "whole U-Net forward (3x3 conv flops / forward time; pool, upsample and head included)",
                     "peak_source": pk["source"] + " bf16_tflops (burst)"},
        "gpu_launches": (6 * L - 3) * ((args.sur_screen + nb - 1) // nb) * args.steps, "clocks": clk.summary(),
    }


def run_stack(args, rank, world, local_rank):
    """The paper's own bump-to-load pipeline on a uniform 4-die stack of 256 x 256 meshes with
    256 TSV columns: 128 bumps on die 0 x 2,048 loads on die 3 (er_stack_pairs: Wu double sums,
    reduced TSV system, LU, m + n solves, pair dots).  Cross-checked, outside the timed region,
    against the sketch route on the same stack (a single pad at one bump, FP64 solve)."""
    import torch
    from paper_2607_05818_gb300 import er
    from paper_2607_05818_gb300 import instances as I

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    M = N = 256
    d, p, m, n = 4, 256, 128, 2048
    rng = np.random.default_rng(20260705 + rank)
    r = np.array([0.05, 0.1, 0.05, 0.1])
    s = r.copy()
    cells = rng.choice(M * N, p, replace=False)
    tsv = np.stack([cells % M, cells // M], axis=1)
    Rt = rng.uniform(0.01, 0.05, (d - 1, p))
    bumps = np.stack([rng.integers(0, M, m), rng.integers(0, N, m)], axis=1)
    loads = np.stack([rng.integers(0, M, n), rng.integers(0, N, n)], axis=1)
    R = torch.empty((m, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        er.stack_pairs(M, N, r, s, tsv, Rt, bumps, loads, R)
    torch.cuda.synchronize()
    stats = []
    with ClockSampler(gpu_index(local_rank)) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(er.stack_pairs(M, N, r, s, tsv, Rt, bumps, loads, R))
        e1.record(stream)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
    n_job, s_max = combine_ranks(m * n, e0.elapsed_time(e1) / 1e3, world, dev)
    value = n_job * args.steps / s_max
    med = {kk: statistics.median(st[kk] for st in stats) for kk in ("ms_wu", "ms_build", "ms_lu", "ms_solve", "ms_dot")}
    wu_flops = 6.0 * stats[-1]["wu_pairs"] * (M - 1) * (N - 1)  # per term: 2 FMA + 2 MUL
    fp64_peak = 1.25  # nominal GB300 FP64 rate (TFLOP/s)
    cs = clk.summary()
    # cross-check: the same stack as a network with one pad (1 ohm) at bump 0; R(bump, load)
    # from the FP64 sketch at k = 256 by er_pair_reff, against row 0 of the paper pipeline
    cross = None
    if rank == 0:
        rx = np.stack([np.full((N, M - 1), r[t]) for t in range(d)])
        ry = np.stack([np.full((N - 1, M), s[t]) for t in range(d)])
        cols = [(t, int(x), int(y), float(Rt[t, j])) for j, (x, y) in enumerate(tsv) for t in range(d - 1)]
        inst = I.from_resistances(rx, ry, cols, [(0, int(bumps[0, 0]), int(bumps[0, 1]), 1.0)], "stack")
        g = er.grid_create(inst)
        kk = 256
        Y = torch.empty((inst.n, kk), dtype=torch.float64, device=dev)
        Z = torch.empty_like(Y)
        er.sketch(g, kk, 7, "fp64", Y)
        er.solve(g, Y, Z, kk, "fp64")
        b0 = int(bumps[0, 1]) * M + int(bumps[0, 0])
        lid = (d - 1) * M * N + loads[:, 1].astype(np.int64) * M + loads[:, 0]
        Rj = torch.empty((1, n), dtype=torch.float64, device=dev)
        er.pair_reff(g, Z, kk, "fp64", [b0], lid, Rj)
        torch.cuda.synchronize()
        a, b = Rj.cpu().numpy()[0], R[0].cpu().numpy()
        rel = np.abs(a / b - 1)
        cross = {"vs": "sketch route (k=256, FP64 solve, er_pair_reff) on the same stack, bump 0 x all loads",
                 "mean_rel_diff": float(rel.mean()), "max_rel_diff": float(rel.max()),
                 "jl_noise_expected": float(np.sqrt(2 / kk))}
        g.destroy()
    peaks = load_peaks()
    cpu = None
    if rank == 0 and world == 1:
        # the oracle's reduced system (long-double Wu sums, LAPACK LU) on a bounded sample of
        # the recipe: 64 x 64 dies, 32 TSV columns, 16 bumps x 128 loads
        from oracle import reduced as ored
        Ms, ps, ms_, ns = 64, 32, 16, 128
        rs = np.random.default_rng(3)
        cs_ = rs.choice(Ms * Ms, ps, replace=False)
        t0 = time.perf_counter()
        ost = ored.UniformStack(Ms, Ms, r, s, [(int(c % Ms), int(c // Ms)) for c in cs_],
                                rs.uniform(0.01, 0.05, (d - 1, ps)))
        ored.TransformedSystem(ost).pairs([tuple(x) for x in rs.integers(0, Ms, (ms_, 2))],
                                          [tuple(x) for x in rs.integers(0, Ms, (ns, 2))])
        dt = time.perf_counter() - t0
        cpu = {"value": ms_ * ns / dt, "unit": "pairs/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle.reduced.TransformedSystem on {d} dies of {Ms}x{Ms}, {ps} TSV columns, "
                         f"{ms_} x {ns} pairs ({dt:.1f} s)"}
    return {
        "metric": "bump-load effective resistances per second, paper pipeline (Wu + reduced TSV system + LU)",
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * s_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "stack_pairs_4x256x256", "dies": d, "mesh": [M, N], "tsv_columns": p, "bumps": m,
                   "loads": n, "system_order": stats[-1]["n_system"], "wu_pairs": stats[-1]["wu_pairs"],
                   "l2": "working set (cosine tables, 1/lambda, reduced system) is L2-resident; FP64-bound"},
        "phase_ms": med,
        "roofline": {"kernel": "k_wu<8> (Eq. 3 double sums)", "bound": "alu",
                     "achieved": wu_flops / (med["ms_wu"] / 1e3) / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": wu_flops / (med["ms_wu"] / 1e3) / 1e12 / fp64_peak, "traffic": None,
                     "flops_per_call": wu_flops, "peak_source": "nominal GB300 FP64 rate (1.25 TFLOP/s)"},
        "cross_check": cross, "cpu_baseline": cpu,
        # per call: 2 cosine tables, d x (1/lambda + Wu), C and RHS, 4 per LU panel (the last
        # panel has no trailing update), the solves and the pair dots
        "gpu_launches": args.steps * (2 + 2 * d + 2 + 4 * -(-stats[-1]["n_system"] // 32) - 2 + 2),
        "clocks": cs, "hbm_peak_gbs": peaks["hbm_gbs"],
    }


def run_planning(args, rank, world, local_rank):
    """TSV-planning sweep (the paper's band-like against uniform TSV plans): 4 uniform tiers of
    256 x 256, 1,024 bumps on an 8-node pitch, four 64 x 32 functional blocks on the top tier
    drawing 1 A each; plans with 512, 1,024 and 2,048 TSV columns as a 32-row band, a 64-row
    band and a uniform grid.  One step = R maps of all 9 plans (batching form, k = 64) + the
    exact IR drop of the load per plan (er_solve, FP32 form) + through-bump currents."""
    import torch
    from paper_2607_05818_gb300 import planning as P

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    plans = [P.floorplan(pat, n_tsv=nt, band_rows=br)
             for nt in (512, 1024, 2048) for pat, br in (("band", 32), ("band", 64), ("uniform", 0))]
    for _ in range(args.warmup):
        P.sweep(plans[:1], k=64, device=dev)
    torch.cuda.synchronize()
    recs = []
    with ClockSampler(gpu_index(local_rank)) as clk:
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            recs.append(P.sweep(plans, k=64, device=dev))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        dt = time.perf_counter() - t0
    n_job, s_max = combine_ranks(len(plans), dt, world, dev)
    res, tm = recs[-1]
    return {
        "metric": "TSV plans analysed per second (R map + exact IR drop + through-bump currents)",
        "value": n_job * args.steps / s_max, "unit": "plans/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * s_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "tsv_planning_4x256x256", "plans": len(plans), "nodes_per_plan": plans[0].n,
                   "bumps": int(len(plans[0].pad_g)), "blocks": 4, "block_current_A": 1.0, "k_maps": 64},
        "timing_s": tm, "plans": res,
        "paper_context": "Sec. IV-B on its own floorplan: 23.4% of bumps carry 95% of the current with a band, "
                         "53.2% with uniform TSVs",
        "roofline": None, "cpu_baseline": None, "gpu_launches": None, "clocks": clk.summary(),
    }


def fp64_accuracy(er, g, inst, k, seed, R, tol32, block, dev, fp32_solve_s):
    """This form's R map against plain FP64 GPU PCG (tol 1e-12) on the same network and seed,
    outside the timed region.  With block > 0 the FP64 reference solves the k sketch columns in
    blocks of `block` (the columns are independent solves; each block's partial map is summed),
    which bounds its memory on the large networks.  Also plain FP64 stopped at this form's
    tolerance, for the speedup at equal accuracy (in block mode measured on the first block and
    scaled to k columns)."""
    import torch
    block = k if block <= 0 or block >= k else block
    Y64 = torch.empty((inst.n, k), dtype=torch.float64, device=dev)
    er.sketch(g, k, seed, "fp64", Y64)
    R64 = torch.zeros(inst.n, dtype=torch.float64, device=dev)
    Rb = torch.empty_like(R64)
    Zb = torch.empty((inst.n, block), dtype=torch.float64, device=dev)
    its, secs, same = [], 0.0, None
    for b0 in range(0, k, block):
        Yb = Y64 if block == k else Y64[:, b0:b0 + block].contiguous()
        _, st = er.solve(g, Yb, Zb, block, "fp64")
        er.reff_map(g, Zb, block, "fp64", Rb)
        R64 += Rb
        its.append(st["iterations"])
        secs += st["seconds"]
        if b0 == 0:  # plain FP64 PCG stopped at the same residual tolerance as this form
            o_same = er.default_solve_opts("fp64")
            o_same.tol = tol32
            Zs = torch.empty_like(Zb)
            _, st_same = er.solve(g, Yb, Zs, block, "fp64", o_same)
            Rs = torch.empty_like(R64)
            er.reff_map(g, Zs, block, "fp64", Rs)
            same = (st_same, Rs.cpu().numpy(), Rb.cpu().numpy())
            del Zs, Rs
        del Yb
    torch.cuda.synchronize()
    a, b = R.cpu().numpy(), R64.cpu().numpy()
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    rel = np.abs(a[fin] / b[fin] - 1)
    st_same, rs, rb = same
    rel_same = np.abs(rs[fin] / rb[fin] - 1)
    same_s = st_same["seconds"] * (k / block)
    return {"vs": "plain FP64 GPU PCG (Jacobi, tol 1e-12), same network and seed", "max_rel_err": float(rel.max()),
            "mean_rel_err": float(rel.mean()), "nodes_compared": int(fin.sum()), "tol": tol32,
            "fp64_ref_iterations": max(its), "fp64_ref_solve_s": secs,
            "fp64_ref_column_blocks": k // block,
            "fp64_same_tol": {"iterations": st_same["iterations"], "solve_s": same_s,
                              "max_rel_err": float(rel_same.max()),
                              "note": "all columns" if block == k else
                              f"measured on the first {block} columns (vs the reference's same columns), "
                              f"time scaled to {k}"},
            "this_form_solve_s": fp32_solve_s, "speedup_vs_fp64_same_tol": same_s / fp32_solve_s}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2607_05818_gb300 import er

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    shard = args.shard == "columns" and world > 1
    inst = make_workload(args.workload, 0 if shard else rank)  # column shards: one network on every rank
    k_total = args.k
    j0, k = er.column_shard(k_total, world, rank) if shard else (0, k_total)
    seed = int(inst.meta.get("seed", 1))
    prec = args.prec
    dt = torch.float32 if prec == "fp32" else torch.float64
    es = 4 if prec == "fp32" else 8
    g = er.grid_create(inst)
    info = g.info()
    n_ok = info["n_nodes"] - info["n_floating"]
    Yt = torch.empty((inst.n, k), dtype=dt, device=dev)
    Z = torch.empty_like(Yt)
    R = torch.empty(inst.n, dtype=torch.float64, device=dev)
    opts = er.default_solve_opts(prec)
    if args.tol is not None:
        opts.tol = args.tol
    mg = prec == "fp32" and args.precond == "mg"
    opts.precond = 1 if mg else 0
    if mg:
        opts.check_every = 2  # a multigrid iteration costs several stencil passes: poll sooner
    opts.profile = 1
    stream = torch.cuda.current_stream()

    def step():
        if shard:
            er.sketch_cols(g, k_total, j0, k, seed, prec, Yt)
        else:
            er.sketch(g, k, seed, prec, Yt)
        _, st = er.solve(g, Yt, Z, k, prec, opts)
        er.reff_map(g, Z, k, prec, R)
        if shard:
            reduce_partial_map(R, world)
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    stats = []
    with ClockSampler(gpu_index(local_rank)) as clk:
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            stats.append(step())
        e1.record(stream)
        barrier()
    # replicas: every rank's network counts; column shards: the one network all ranks mapped
    n_total, s_max = combine_ranks(n_ok if (not shard or rank == 0) else 0, e0.elapsed_time(e1) / 1e3, world, dev)
    ms = 1e3 * s_max
    value = n_total * args.steps / s_max

    # per-pass durations measured live (CUDA events on the solver stream) in the timed region
    launches = np.sum([s["launches"] for s in stats], axis=0)
    kms = np.sum([s["kernel_ms"] for s in stats], axis=0)
    iters = [s["iterations"] for s in stats]
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else None
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    peak_note = "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s"
    nk = inst.n * k
    coef = 16 * inst.n  # per-node coefficient words read by a stencil pass
    if mg:
        # (pass kind index, kernel, algorithmic bytes per launch).  Finest level: the restriction
        # reads r and writes r_1 (n/4 rows); the post-sweep reads r and z_1 and writes z.  The
        # coarse levels together (pass kind 5, one entry per V-cycle) move 3.5 n_l k s per level,
        # n_l = n / 4^l for l >= 1, a factor 1/3 of the finest level's 3.5 n k s.
        kinds = [(1, "k_mg_upd_tile<true>", 6 * nk * es + coef),    # p', r, x, p'_prev in; r, x out
                 (4, "k_mg_upd_tile<false>", 3 * nk * es + coef),   # p', r in; r out
                 (0, "k_mg_dir_tile", 3 * nk * es + coef),          # z, p in; p' out
                 (7, "k_mg_tile<true, true> (finest level)", int(2.25 * nk * es) + coef),
                 (6, "k_mg_tile<false, false> (finest level)", int(1.25 * nk * es) + coef),
                 (5, "V-cycle on the coarse levels", int(3.5 * nk * es / 3)),
                 (2, "k_tma<MODE_R> (double-float residual)", 4 * nk * es + coef)]  # x {hi, lo}, b in; r out
    elif prec == "fp32":
        # (pass kind index, kernel, algorithmic bytes per launch)
        kinds = [(1, "k_tma<MODE_B>", 6 * nk * es + coef),   # odd iterations: r, p, x in; x, r, p' out
                 (4, "k_tma<MODE_B0>", 4 * nk * es + coef),  # even iterations: r, p in; r, p' out
                 (0, "k_tma<MODE_A_DOT>", 2 * nk * es + coef),  # r, p in
                 (2, "k_tma<MODE_R> (double-float residual)", 4 * nk * es + coef)]  # x {hi, lo}, b in; r out
    else:
        kinds = [(0, "k_stencil<double,double,MODE_A_STORE>", 4 * nk * es + coef),
                 (1, "k_stream<double,MODE_S>", 6 * nk * es)]
    rl = []
    n_levels = None
    if mg:
        n_levels = 1  # the library coarsens 2 x 2 per tier until a level has at most 1,024 nodes
        Wl, Hl = inst.W, inst.H
        while inst.T * Wl * Hl > 1024 and max(Wl, Hl) > 1:
            Wl, Hl, n_levels = (Wl + 1) // 2, (Hl + 1) // 2, n_levels + 1
    for idx, name, nbytes in kinds:
        n_l = int(launches[idx])
        if idx == 5:  # coarse-level launches of one V-cycle: down and up per level pair below
            n_l = n_l // max(1, 2 * n_levels - 3)  # the finest, plus the coarsest level
        avg_ms = float(kms[idx]) / max(n_l, 1)
        ach = nbytes / (avg_ms / 1e3) / 1e9 if avg_ms > 0 else None
        rl.append({"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                   "frac": (ach / peak) if ach else None, "traffic": ncu_traffic(name, args.workload),
                   "algorithmic_bytes_per_launch": nbytes, "avg_launch_ms": avg_ms, "launches": n_l,
                   "share_of_step": float(kms[idx]) / ms if ms > 0 else None, "peak_source": peak_note})
    rl.sort(key=lambda r: -(r["share_of_step"] or 0))
    pass_names = ["A", "B", "R", "other", "B0", "MG", "MG_down0", "MG_up0"]
    pass_ms_per_step = {pass_names[i]: float(kms[i]) / args.steps for i in range(len(kms))}
    gpu_launches = int(launches.sum()) + 2 * args.steps  # + sketch and reff_map per step

    result = {"rank0_iterations": iters, "stats_last": stats[-1], "pass_ms_per_step": pass_ms_per_step,
              "replacements": [s["sweeps"] for s in stats],
              "max_rel_residual": max(s["max_rel_residual"] for s in stats)}
    acc = None
    if rank == 0 and not args.no_accuracy and prec == "fp32":
        acc = fp64_accuracy(er, g, inst, k_total, seed, R, opts.tol, args.acc_block, dev,
                            float(np.median([s["seconds"] for s in stats])))
    # end to end through the host entry point: host arrays in, host R out (copies inside)
    e2e = None
    if rank == 0:
        opts_e = er.default_solve_opts(prec)
        opts_e.precond = opts.precond
        opts_e.check_every = opts.check_every
        if args.tol is not None:
            opts_e.tol = opts.tol
        R_host = np.empty(inst.n)
        t0 = time.perf_counter()
        er.reff_map_host(inst, k_total, seed, prec, opts_e, R_host)
        e2e_s = time.perf_counter() - t0
        e2e = {"value": n_ok / e2e_s, "unit": UNIT, "h2d_bytes_per_step": info["h2d_bytes"],
               "d2h_bytes_per_step": inst.n * 8, "seconds": e2e_s,
               "note": "er_reff_map_host: host assembly + H2D + sketch + solve + map + D2H of R"}
    return value, ms, result, rl, gpu_launches, clk.summary(), acc, e2e, n_total


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))

    if args.impl == "reference":
        # the reference arm is the CPU oracle as it stands, rank 0 only
        if rank != 0:
            return
        from oracle import build as ob
        ob.build()
        inst = cpu_sample_instance(args.cpu_sample)
        for _ in range(args.warmup):
            oracle_step(inst, args.k, 1)
        ts, phases = [], []
        n_ok, thr = 0, 1
        for _ in range(args.steps):
            ph, n_ok, thr = oracle_step(inst, args.k, 1)
            ts.append(ph["total_s"])
            phases.append(ph)
        tot = sum(ts)
        v = n_ok * args.steps / tot
        print(json.dumps({
            "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "k": args.k,
                                            "sample": f"{inst.T}x{inst.W}x{inst.H}"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle", "cpu_model": cpu_model(),
                             "nproc": os.cpu_count(),
                             "sample": f"one {inst.T}x{inst.W}x{inst.H} network of the same recipe per step "
                                       f"(SuperLU factorisation, C sketch, {args.k} solves on {thr} threads, row norms)",
                             "phases_s_last_step": {k_: round(v_, 3) for k_, v_ in phases[-1].items()} if phases else None},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    special = {"batch_candidates": run_batch, "surrogate": run_surrogate, "pairs": run_pairs,
               "unet_forward": run_unet_forward, "stack_pairs": run_stack, "tsv_planning": run_planning}
    run = next((f for pre, f in special.items() if args.workload.startswith(pre)), None)
    if run is not None:
        line = run(args, rank, world, local_rank)
        if rank == 0:
            print(json.dumps(line))
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    value, ms, result, rl, launches, clocks, acc, e2e, n_total = run_ours(args, rank, world, local_rank)
    if rank == 0:
        cpu = cpu_baseline(args) if world == 1 else None
        sharded = args.shard == "columns" and world > 1
        n_rank = n_total if sharded else int(n_total / world)  # nodes each rank's arrays hold
        k_rank = args.k // world if sharded else args.k
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if (args.shard == "columns" and world > 1) else "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.prec == "fp32" else "f64", "data": "synthetic",
            "config": {"workload": args.workload, "k": args.k, "precision": args.prec,
                       "nodes_per_rank": n_rank,
                       "parallelism": (f"column shards: one network, {args.k} sketch columns split over {world} ranks, "
                                       f"partial maps summed by one all-reduce" if args.shard == "columns" and world > 1
                                       else f"replicas: {world} independent network(s), no collective on the data path"),
                       "preconditioner": "aggregation multigrid V-cycle" if (args.precond == "mg" and args.prec == "fp32")
                       else "Jacobi",
                       "l2": f"inputs larger than L2 (each [n][k] array is "
                             f"{n_rank * k_rank * (4 if args.prec == 'fp32' else 8) / 2**30:.2f} GiB)",
                       "iterations_per_step": result["rank0_iterations"],
                       "fp64_residual_replacements_per_step": result["replacements"],
                       "tol": args.tol if args.tol is not None else ("1e-7" if args.prec == "fp32" else "1e-12"),
                       "final_max_rel_residual": result["max_rel_residual"],
                       "kernel_ms_per_step_by_pass": result["pass_ms_per_step"]},
            "roofline": rl[0], "roofline_other": rl[1:], "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks, "accuracy": acc,
        }
        print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
