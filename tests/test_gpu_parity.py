"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Sketch: element by element against the oracle's FP64 sketch.  Solve + map: the FP64
path against the oracle's same-seed JL estimate (dense Cholesky solves) within 1e-9
relative, the FP32+refinement path within 1e-3 relative; ragged sizes, ragged RHS
blocks, floating nodes, a single node and the host-buffer entry point.  The full-size
workloads are in test_gpu_fullsize.py.
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


DEV = "cuda"
F64 = torch.float64
F32 = torch.float32


def gpu_map(er, inst, k, seed, prec, opts=None):
    g = er.grid_create(inst)
    dt = F64 if prec == "fp64" else F32
    Yt = torch.empty((inst.n, k), dtype=dt, device=DEV)
    Z = torch.empty_like(Yt)
    R = torch.empty(inst.n, dtype=F64, device=DEV)
    er.sketch(g, k, seed, prec, Yt)
    _, st = er.solve(g, Yt, Z, k, prec, opts)
    er.reff_map(g, Z, k, prec, R)
    torch.cuda.synchronize()
    out = (Yt.cpu().numpy().astype(np.float64), Z.cpu().numpy().astype(np.float64), R.cpu().numpy(), st)
    g.destroy()
    return out


def rel_err(a, b):
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    return float(np.max(np.abs(a[fin] - b[fin]) / np.abs(b[fin]))) if fin.any() else 0.0


CASES = [
    ("tiny_plain", lambda: I.tiny_plain(), 128),
    ("ragged_3x37x23_k36", lambda: I.random_small(np.random.default_rng(1), T=3, W=37, H=23, n_tsv=40, n_pads=3), 36),
    ("ragged_2x61x70_k4", lambda: I.random_small(np.random.default_rng(2), T=2, W=61, H=70, n_tsv=25, n_pads=2), 4),
    ("floating_1x20x19", lambda: I.random_small(np.random.default_rng(3), T=1, W=20, H=19, n_pads=1,
                                                  open_frac=0.35), 20),
    ("single_node", lambda: I.uniform(1, 1, 1, 1.0, 1.0, pads=[(0, 0, 0, 0.5)]), 8),
    ("chain_1x97", lambda: I.random_small(np.random.default_rng(4), T=1, W=97, H=1, n_pads=1), 12),
    ("small_2x5x3_tsv", lambda: I.random_small(np.random.default_rng(5), T=2, W=5, H=3, n_tsv=4, n_pads=1), 32),
    ("small_1x5x8", lambda: I.random_small(np.random.default_rng(6), T=1, W=5, H=8, n_pads=1), 8),
]


@pytest.mark.parametrize("name,make,k", CASES, ids=[c[0] for c in CASES])
def test_sketch_matches_oracle(er, name, make, k):
    inst = make()
    seed = 777
    ref = osk.sketch_numpy(inst, k, seed)
    g = er.grid_create(inst)
    for prec, dt in (("fp64", F64), ("fp32", F32)):
        Yt = torch.full((inst.n, k), float("nan"), dtype=dt, device=DEV)
        er.sketch(g, k, seed, prec, Yt)
        got = Yt.cpu().numpy().astype(np.float64)
        if prec == "fp64":
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14 * max(1.0, np.abs(ref).max()))
        else:
            np.testing.assert_allclose(got, ref.astype(np.float32).astype(np.float64), rtol=1.2e-7, atol=1e-30)
    g.destroy()


@pytest.mark.parametrize("name,make,k", CASES, ids=[c[0] for c in CASES])
def test_fp64_map_matches_oracle(er, name, make, k):
    inst = make()
    seed = 20260701
    Yt_ref = osk.sketch_numpy(inst, k, seed)
    R_ref, Z_ref = osk.reff_jl_dense(inst, k, seed, Yt_ref)
    _, Z, R, st = gpu_map(er, inst, k, seed, "fp64")
    assert rel_err(R, R_ref) <= 1e-9, (name, rel_err(R, R_ref), st)
    # Z element by element, relative to each column's scale
    colscale = np.maximum(np.abs(Z_ref).max(axis=0), 1e-300)
    assert np.max(np.abs(Z - Z_ref) / colscale) <= 1e-9
    assert st["converged_cols"] == k and st["max_rel_residual"] <= 1e-11
    fl = network.floating_mask(inst)
    assert np.all(np.isinf(R[fl])) and np.all(Z[fl] == 0.0)


@pytest.mark.parametrize("name,make,k", CASES, ids=[c[0] for c in CASES])
def test_fp32_refine_map_within_1e3(er, name, make, k):
    inst = make()
    seed = 31337
    R_ref, _ = osk.reff_jl_dense(inst, k, seed)
    _, _, R, st = gpu_map(er, inst, k, seed, "fp32")
    err = rel_err(R, R_ref)
    assert err <= 1e-3, (name, err, st)
    assert st["max_rel_residual"] <= 1e-7 and st["converged_cols"] == k, (name, st)


def test_tiny_plain_exact_and_jl_report(er):
    """The tiny plain workload: GPU FP64 vs the same-seed oracle (acceptance 1e-9) and the JL
    error against exact diag(G^-1) reported (about sqrt(2/k) per node)."""
    inst = I.tiny_plain()
    k, seed = 128, 20260701
    R_jl, _ = osk.reff_jl_dense(inst, k, seed)
    R_ex = exact.reff_dense(inst)
    _, _, R, st = gpu_map(er, inst, k, seed, "fp64")
    assert rel_err(R, R_jl) <= 1e-9
    jl = np.abs(R / R_ex - 1)
    print(f"JL vs exact: max {jl.max():.3f} mean {jl.mean():.3f} sqrt(2/k) {np.sqrt(2 / k):.3f}; "
          f"iterations {st['iterations']}")
    assert jl.mean() < 1.5 * np.sqrt(2 / k)


def test_host_entry_point_matches_device_path(er):
    inst = I.random_small(np.random.default_rng(9), T=2, W=33, H=31, n_tsv=30, n_pads=4)
    k, seed = 32, 5
    R_dev = gpu_map(er, inst, k, seed, "fp64")[2]
    R_host, st = er.reff_map_host(inst, k, seed, "fp64")
    np.testing.assert_array_equal(R_host, R_dev)
    R32, st32 = er.reff_map_host(inst, k, seed, "fp32")
    assert rel_err(R32, R_dev) <= 1e-3


def test_deterministic_runs(er):
    inst = I.random_small(np.random.default_rng(10), T=2, W=45, H=40, n_tsv=30, n_pads=3)
    a = gpu_map(er, inst, 64, 3, "fp32")[2]
    b = gpu_map(er, inst, 64, 3, "fp32")[2]
    np.testing.assert_array_equal(a, b)


def test_invalid_device_arguments(er):
    inst = I.tiny_plain()
    g = er.grid_create(inst)
    Yt = torch.empty((inst.n, 130), dtype=F64, device=DEV)
    with pytest.raises(er.ErError):
        er.sketch(g, 130, 1, "fp64", Yt)  # k not a multiple of 4
    buf = torch.empty(inst.n * 128 * 8 + 64, dtype=torch.uint8, device=DEV)
    with pytest.raises(er.ErError):
        er.sketch(g, 128, 1, "fp64", buf.data_ptr() + 8)  # not 16-byte aligned
    Z = torch.empty((inst.n, 128), dtype=F64, device=DEV)
    Y = torch.zeros((inst.n, 128), dtype=F64, device=DEV)
    with pytest.raises(er.ErError):
        er.solve(g, Y, Y, 128, "fp64")  # aliasing
    # maxit too small -> ER_ERR_NOT_CONVERGED, reported not raised when allowed
    er.sketch(g, 128, 1, "fp64", Y)
    s, st = er.solve(g, Y, Z, 128, "fp64", er.default_solve_opts("fp64", maxit=3), allow_unconverged=True)
    assert s == er.ER_ERR_NOT_CONVERGED and st["iterations"] == 3
    g.destroy()


def test_column_shards_sum_to_the_map(er):
    """Column sharding of one network (the multi-GPU partition): each shard's sketch columns are
    bitwise the same columns of the whole sketch, and the shards' partial maps add up to the
    whole map.  The shards run one after another on one GPU; across GPUs the sum is one
    all-reduce of the n-vector."""
    inst = I.random_small(np.random.default_rng(31), T=3, W=37, H=23, n_tsv=40, n_pads=3, open_frac=0.1)
    k, seed, world = 48, 123, 3
    for prec, dt in (("fp64", F64), ("fp32", F32)):
        Y_full, _, R_full, _ = gpu_map(er, inst, k, seed, prec)
        g = er.grid_create(inst)
        R_sum = np.zeros(inst.n)
        for rank in range(world):
            j0, kl = er.column_shard(k, world, rank)
            Yt = torch.empty((inst.n, kl), dtype=dt, device=DEV)
            Z = torch.empty_like(Yt)
            R = torch.empty(inst.n, dtype=F64, device=DEV)
            er.sketch_cols(g, k, j0, kl, seed, prec, Yt)
            er.solve(g, Yt, Z, kl, prec)
            er.reff_map(g, Z, kl, prec, R)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(Yt.cpu().numpy().astype(np.float64), Y_full[:, j0:j0 + kl])
            R_sum += R.cpu().numpy()
        g.destroy()
        tol = 1e-12 if prec == "fp64" else 1e-3
        assert rel_err(R_sum, R_full) <= tol, (prec, rel_err(R_sum, R_full))
