"""The batching form through the C ABI: many uneven networks in shared launches must give
each network's R map as the oracle's same-seed JL estimate does (network c uses seed + c),
and agree with the single-network FP32 solve."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import network
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


def make_batch():
    rng = np.random.default_rng(77)
    nets = [I.random_small(rng, T=2, W=37, H=23, n_tsv=30, n_pads=3),
            I.random_small(rng, T=3, W=64, H=64, n_tsv=60, n_pads=4),
            I.random_small(rng, T=1, W=20, H=19, n_pads=1, open_frac=0.35),
            I.random_small(rng, T=2, W=5, H=3, n_tsv=4, n_pads=1),
            I.batch_candidate(rng, 4, T=2, W=64, n_tsv=50, clustered=True),
            I.random_small(rng, T=4, W=33, H=70, n_tsv=80, n_pads=2)]
    return nets


def test_batch_matches_oracle_and_single_solve(er):
    nets = make_batch()
    k, seed = 32, 4242
    grids = [er.grid_create(n) for n in nets]
    R = [torch.empty(n.n, dtype=torch.float64, device="cuda") for n in nets]
    s, st = er.batch_solve(grids, k, seed, R, tile_rows=[0, 32, 0, 0, 64, 16])
    torch.cuda.synchronize()
    assert st["n_grids"] == len(nets) and st["converged"] == len(nets)
    assert st["graph_captures"] >= 1
    for c, (net, g) in enumerate(zip(nets, grids)):
        ref, _ = osk.reff_jl_dense(net, k, seed + c)
        got = R[c].cpu().numpy()
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(got), fin)
        assert np.all(np.isinf(got[network.floating_mask(net)]))
        err = np.max(np.abs(got[fin] / ref[fin] - 1)) if fin.any() else 0.0
        assert err <= 1e-3, (c, err)
        # the single-network FP32 solve on the same sketch
        Y = torch.empty((net.n, k), dtype=torch.float32, device="cuda")
        Z = torch.empty_like(Y)
        R1 = torch.empty(net.n, dtype=torch.float64, device="cuda")
        er.sketch(g, k, seed + c, "fp32", Y)
        er.solve(g, Y, Z, k, "fp32")
        er.reff_map(g, Z, k, "fp32", R1)
        torch.cuda.synchronize()
        one = R1.cpu().numpy()
        if fin.any():
            assert np.max(np.abs(got[fin] / one[fin] - 1)) <= 1e-4, c
    for g in grids:
        g.destroy()


def test_batch_rejects_fp64_and_bad_args(er):
    nets = make_batch()[:2]
    grids = [er.grid_create(n) for n in nets]
    R = [torch.empty(n.n, dtype=torch.float64, device="cuda") for n in nets]
    with pytest.raises(er.ErError):
        er.batch_solve(grids, 32, 1, R, prec="fp64")
    with pytest.raises(er.ErError):
        er.batch_solve(grids, 30, 1, R)
    for g in grids:
        g.destroy()


def test_multigrid_batch_equals_single_solves(er):
    """precond = 1: every pass of the multigrid iteration is one persistent launch over all
    running networks, each block running er_solve's kernel body, and the loop's decisions are
    er_solve's; so each map is bitwise the map of sketch + solve + map on that network alone,
    and within the FP32 form's bound of the oracle.  Networks too small for a hierarchy (the
    5 x 3 and 20 x 19 ones) take er_solve's Jacobi path, as alone."""
    nets = make_batch()
    k, seed = 32, 515
    grids = [er.grid_create(n) for n in nets]
    R = [torch.full((n.n,), float("nan"), dtype=torch.float64, device="cuda") for n in nets]
    opts = er.default_solve_opts("fp32", precond=1, check_every=2)
    s, st = er.batch_solve(grids, k, seed, R, opts=opts)
    torch.cuda.synchronize()
    assert st["n_grids"] == len(nets) and st["converged"] == len(nets)
    assert st["nodes"] == sum(n.n - int(network.floating_mask(n).sum()) for n in nets)
    for c, (net, g) in enumerate(zip(nets, grids)):
        Y = torch.empty((net.n, k), dtype=torch.float32, device="cuda")
        Z = torch.empty_like(Y)
        R1 = torch.empty(net.n, dtype=torch.float64, device="cuda")
        er.sketch(g, k, seed + c, "fp32", Y)
        er.solve(g, Y, Z, k, "fp32", opts)
        er.reff_map(g, Z, k, "fp32", R1)
        torch.cuda.synchronize()
        got, one = R[c].cpu().numpy(), R1.cpu().numpy()
        assert np.array_equal(got, one), c  # +inf at floating nodes compares equal
        ref, _ = osk.reff_jl_dense(net, k, seed + c)
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(got), fin)
        if fin.any():
            assert np.max(np.abs(got[fin] / ref[fin] - 1)) <= 1e-3, c
    for g in grids:
        g.destroy()


def test_multigrid_autotuned_order_is_valid_and_changes_only_speed(er, tmp_path, monkeypatch):
    """The autotuner's choice of the multigrid kernels' launch order, per size class, is one of
    its candidates, and the maps it gives are bitwise those of the library's default, both for
    er_solve and for the batching form."""
    monkeypatch.setenv("ER_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_2607_05818_gb300 import autotune
    rng = np.random.default_rng(2025)
    nets = [I.batch_candidate(rng, 0, T=2, W=64, n_tsv=60), I.batch_candidate(rng, 1, T=3, W=128, n_tsv=200),
            I.batch_candidate(rng, 2, T=4, W=64, n_tsv=100, clustered=True)]
    k, seed = 64, 99
    orders = [autotune.best_mg_order(n, k) for n in nets]
    print(f"tuned orders {orders}; timings {autotune._load()}")
    assert all(o in autotune.CANDIDATE_MG_ORDERS for o in orders)
    grids = [er.grid_create(n) for n in nets]
    opts = er.default_solve_opts("fp32", precond=1, check_every=2)
    R0 = [torch.empty(n.n, dtype=torch.float64, device="cuda") for n in nets]
    R1 = [torch.empty(n.n, dtype=torch.float64, device="cuda") for n in nets]
    R2 = [torch.empty(n.n, dtype=torch.float64, device="cuda") for n in nets]
    er.batch_solve(grids, k, seed, R0, opts=opts)
    er.batch_solve(grids, k, seed, R1, opts=opts, tile_rows=orders)
    er.batch_solve(grids, k, seed, R2, opts=opts, tile_rows=[3 - o for o in orders])
    torch.cuda.synchronize()
    for a, b, c in zip(R0, R1, R2):
        assert torch.equal(a, b) and torch.equal(a, c)
    # er_solve with each launch order: the same map
    net, g = nets[1], grids[1]
    Y = torch.empty((net.n, k), dtype=torch.float32, device="cuda")
    er.sketch(g, k, seed, "fp32", Y)
    outs = []
    for o in autotune.CANDIDATE_MG_ORDERS:
        Z = torch.empty_like(Y)
        er.solve(g, Y, Z, k, "fp32", er.default_solve_opts("fp32", precond=1, check_every=2, block_order=o))
        outs.append(Z)
    torch.cuda.synchronize()
    for Z in outs[1:]:
        assert torch.equal(Z, outs[0])
    for g in grids:
        g.destroy()
