"""Full-size parity of the FP32 form as the bench runs it (multigrid V-cycle preconditioner,
polled every 2 iterations) and of its Jacobi variant.

4 x 512 x 512, k = 256: Z rows (all 256 columns, so every RHS column block) and R at a few
hundred nodes chosen to cover every class of node the kernels treat differently -- the
edges of the stencil and multigrid tiles in x and y, the first and last rows of every tier,
every TSV node and pad around one TSV cluster, mesh corners -- against the oracle's exact
sparse solves with the same sketch.

8 x 1024 x 1024 (10% of the segments open, floating islands), k = 256: the oracle cannot
factor this network, so the FP32 form is compared with the GPU's plain FP64 form on every
node.  Columns are independent solves and column j of the sketch does not depend on k other
than through the 1/sqrt(k) scale, so the FP64 form solves the first 8 columns (a k = 8
sketch, scaled) and every node's partial map over those columns is compared; floating nodes
must be exactly excluded.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import exact, network
from oracle import sketch as osk
from paper_2607_05818_gb300 import instances as I


@pytest.fixture(scope="module")
def er():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_05818_gb300 import er as mod
    return mod


def class_nodes(inst, rng):
    """Node ids covering the node classes of the 4 x 512 x 512 network, with a label each."""
    T, W, H = inst.T, inst.W, inst.H
    nid = lambda t, y, x: int(network.node_id(T, W, H, t, y, x))
    out = {}
    # stencil passes: 30 owned + 2 halo nodes along x; multigrid tiles: 32 x 8 (restriction,
    # prolongation) and 32 x 4 (CG passes) nodes; 2 x 2 aggregates
    xs = [0, 1, 2, 29, 30, 31, 32, 33, 59, 60, 63, 64, 65, W // 2 - 1, W // 2, W - 3, W - 2, W - 1]
    ys = [0, 1, 3, 4, 7, 8, 9, 63, 64, H // 2, H - 2, H - 1]
    for t in range(T):
        for x, y in zip(rng.choice(xs, 16), rng.choice(ys, 16)):
            out[nid(t, int(y), int(x))] = "tile edge"
        for y in (0, H - 1):                                   # first / last row of the tier
            out[nid(t, y, int(rng.integers(0, W)))] = "tier row"
        for y, x in ((0, 0), (0, W - 1), (H - 1, 0), (H - 1, W - 1)):
            out[nid(t, y, x)] = "corner"
    # every TSV node and pad around the first TSV column's cluster
    x0, y0 = int(inst.tsv_x[0]), int(inst.tsv_y[0])
    near = (np.abs(inst.tsv_x - x0) <= 16) & (np.abs(inst.tsv_y - y0) <= 16)
    for t, x, y in zip(inst.tsv_tier[near], inst.tsv_x[near], inst.tsv_y[near]):
        out[nid(int(t), int(y), int(x))] = "TSV"
        out[nid(int(t) + 1, int(y), int(x))] = "TSV"
    pn = (np.abs(inst.pad_x - x0) <= 24) & (np.abs(inst.pad_y - y0) <= 24)
    for t, x, y in zip(inst.pad_tier[pn], inst.pad_x[pn], inst.pad_y[pn]):
        out[nid(int(t), int(y), int(x))] = "pad"
    for i in rng.integers(0, inst.n, 48):
        out.setdefault(int(i), "random")
    nodes = np.array(sorted(out))
    return nodes, [out[i] for i in nodes]


@pytest.fixture(scope="module")
def precision_oracle():
    inst = I.precision_4x512()
    k, seed = 256, inst.meta["seed"]
    nodes, labels = class_nodes(inst, np.random.default_rng(12))
    Yt_ref = osk.sketch(inst, k, seed)
    f = exact.SparseFactor(inst)
    # Z_i = (G^-1 e_i)^T Y^T for every sampled node: a block of unit right-hand sides
    E = np.zeros((inst.n, len(nodes)))
    E[nodes, np.arange(len(nodes))] = 1.0
    Gi = f.solve(E)
    Z_ref = Gi.T @ Yt_ref
    return inst, k, seed, nodes, labels, Yt_ref[nodes], Z_ref


@pytest.mark.parametrize("precond", [1, 0], ids=["multigrid", "jacobi"])
def test_precision_workload_node_classes(er, precision_oracle, precond):
    inst, k, seed, nodes, labels, Yt_rows, Z_ref = precision_oracle
    g = er.grid_create(inst)
    Yt = torch.empty((inst.n, k), dtype=torch.float32, device="cuda")
    Z = torch.empty_like(Yt)
    R = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    er.sketch(g, k, seed, "fp32", Yt)
    opts = er.default_solve_opts("fp32", precond=precond, check_every=2 if precond else 10)
    _, st = er.solve(g, Yt, Z, k, "fp32", opts)
    er.reff_map(g, Z, k, "fp32", R)
    torch.cuda.synchronize()
    idx = torch.as_tensor(nodes, device="cuda")
    Ys = Yt[idx].double().cpu().numpy()
    Zs = Z[idx].double().cpu().numpy()
    Rs = R[idx].cpu().numpy()
    g.destroy()
    np.testing.assert_allclose(Ys, Yt_rows.astype(np.float32).astype(np.float64), rtol=1.2e-7, atol=0)
    R_ref = np.sum(Z_ref * Z_ref, axis=1)
    rms = np.sqrt(R_ref / k)
    ez = np.max(np.abs(Zs - Z_ref), axis=1) / rms            # per node, over all 256 columns
    er_ = np.abs(Rs / R_ref - 1)
    for cls in sorted(set(labels)):
        m = np.array([lb == cls for lb in labels])
        print(f"{cls:10s} {m.sum():4d} nodes: R max rel err {er_[m].max():.2e}, Z max err / rms {ez[m].max():.2e}")
    print(f"precond {precond}: {len(nodes)} nodes, iterations {st['iterations']}, "
          f"max rel residual {st['max_rel_residual']:.2e}")
    assert len(nodes) >= 200
    assert er_.max() <= 1e-3
    assert ez.max() <= 1e-3
    assert st["converged_cols"] == k and st["max_rel_residual"] <= 1e-7


def test_large_workload_against_fp64_every_node(er):
    """8 x 1024 x 1024, k = 256, the FP32 form with the multigrid preconditioner as the bench
    runs it, against the plain FP64 form on the first 8 sketch columns at every node; sketch
    rows at sampled nodes against the oracle; R against the row norms of Z; floating nodes."""
    inst = I.large_8x1024()
    k, seed, kc = 256, inst.meta["seed"], 8
    g = er.grid_create(inst)
    Yt = torch.empty((inst.n, k), dtype=torch.float32, device="cuda")
    Z = torch.empty_like(Yt)
    R = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    er.sketch(g, k, seed, "fp32", Yt)
    _, st = er.solve(g, Yt, Z, k, "fp32", er.default_solve_opts("fp32", precond=1, check_every=2))
    er.reff_map(g, Z, k, "fp32", R)
    Y64 = torch.empty((inst.n, kc), dtype=torch.float64, device="cuda")
    Z64 = torch.empty_like(Y64)
    er.sketch(g, kc, seed, "fp64", Y64)
    _, st64 = er.solve(g, Y64, Z64, kc, "fp64", er.default_solve_opts("fp64", maxit=60000))
    torch.cuda.synchronize()
    scale = float(np.sqrt(k / kc))
    z32 = Z[:, :kc].double() * scale                      # the same columns on the k = 8 scale
    fl = torch.as_tensor(network.floating_mask(inst), device="cuda")
    assert torch.all(torch.isinf(R[fl])) and torch.all(torch.isfinite(R[~fl]))
    assert torch.all(Z[fl] == 0) and torch.all(Z64[fl] == 0)
    r32 = (z32 * z32).sum(1)[~fl]
    r64 = (Z64 * Z64).sum(1)[~fl]
    rel = (r32 / r64 - 1).abs()
    ez = ((z32 - Z64).abs().amax(1)[~fl] / (r64 / kc).sqrt())
    print(f"large: FP32 multigrid {st['iterations']} iterations; FP64 {st64['iterations']} iterations; "
          f"partial R over {kc} columns at {int((~fl).sum())} nodes: max rel err {rel.max().item():.2e}, "
          f"mean {rel.mean().item():.2e}; Z max err / rms {ez.max().item():.2e}; "
          f"{int(fl.sum())} floating nodes")
    assert rel.max().item() <= 1e-3
    assert ez.max().item() <= 1e-3
    # sketch rows and R at sampled nodes, including floating-island borders
    rng = np.random.default_rng(8)
    T, W, H = inst.T, inst.W, inst.H
    floating = fl.cpu().numpy()
    border = np.flatnonzero(~floating & (np.roll(floating, 1) | np.roll(floating, -1)))
    special = [0, inst.n - 1, W - 1, (T - 1) * W * H + (H - 1) * W,
               int(network.node_id(T, W, H, inst.tsv_tier[0], inst.tsv_y[0], inst.tsv_x[0])),
               int(network.node_id(T, W, H, inst.pad_tier[3], inst.pad_y[3], inst.pad_x[3])),
               int(np.flatnonzero(floating)[0])]
    nodes = np.unique(np.concatenate([rng.integers(0, inst.n, 24), special, rng.choice(border, 16)]))
    idx = torch.as_tensor(nodes, device="cuda")
    Ys, Zs, Rh = Yt[idx].double().cpu().numpy(), Z[idx].double().cpu().numpy(), R[idx].cpu().numpy()
    np.testing.assert_allclose(Ys, osk.sketch_rows(inst, nodes, k, seed).astype(np.float32).astype(np.float64),
                               rtol=1.2e-7, atol=0)
    fin = np.isfinite(Rh)
    np.testing.assert_allclose(Rh[fin], np.sum(Zs[fin] ** 2, axis=1), rtol=1e-12)
    assert st["max_rel_residual"] <= 1e-7 and st64["converged_cols"] == kc
    g.destroy()
