"""The FP32 form with the aggregation-multigrid preconditioner (er_solve_opts.precond = 1)
against the oracle's same-seed JL estimate.

The preconditioner changes only the path to the solution: a column still stops when its
accurate (double-float) residual meets tol, so the maps must meet the FP32 form's bound (1e-3 relative)
against the oracle on every case the Jacobi path is tested on, plus networks whose
coarsening is uneven (odd W and H, a 1 x L chain, floating islands that must stay out of
every aggregate).  On the precision recipe the V-cycle must cut the iteration count by a
large factor, and repeated runs must be bitwise identical.
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


def run(er, inst, k, seed, precond, **over):
    g = er.grid_create(inst)
    Yt = torch.empty((inst.n, k), dtype=torch.float32, device="cuda")
    Z = torch.empty_like(Yt)
    R = torch.empty(inst.n, dtype=torch.float64, device="cuda")
    er.sketch(g, k, seed, "fp32", Yt)
    _, st = er.solve(g, Yt, Z, k, "fp32", er.default_solve_opts("fp32", precond=precond, **over))
    er.reff_map(g, Z, k, "fp32", R)
    torch.cuda.synchronize()
    out = R.cpu().numpy(), st
    g.destroy()
    return out


def rel_err(a, b):
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    return float(np.max(np.abs(a[fin] - b[fin]) / np.abs(b[fin]))) if fin.any() else 0.0


CASES = [
    ("tiny_plain_2x32x32", lambda: I.tiny_plain(), 128),
    ("ragged_3x37x23_k36", lambda: I.random_small(np.random.default_rng(1), T=3, W=37, H=23, n_tsv=40, n_pads=3), 36),
    ("ragged_2x61x70_k4", lambda: I.random_small(np.random.default_rng(2), T=2, W=61, H=70, n_tsv=25, n_pads=2), 4),
    ("floating_1x40x39", lambda: I.random_small(np.random.default_rng(3), T=1, W=40, H=39, n_pads=2,
                                                 open_frac=0.3), 20),
    ("chain_1x97", lambda: I.random_small(np.random.default_rng(4), T=1, W=97, H=1, n_pads=1), 12),
    ("column_5x1x45", lambda: I.random_small(np.random.default_rng(7), T=5, W=1, H=45, n_tsv=12, n_pads=1), 8),
    ("precision_4x96x80", lambda: I.precision_4x512(W=96, H=80, n_tsv=60, n_clusters=3), 64),
]


@pytest.mark.parametrize("name,make,k", CASES, ids=[c[0] for c in CASES])
def test_mg_map_matches_oracle(er, name, make, k):
    inst = make()
    seed = 4242
    R_ref, _ = osk.reff_jl_dense(inst, k, seed)
    R, st = run(er, inst, k, seed, 1)
    err = rel_err(R, R_ref)
    assert err <= 1e-3, (name, err, st)
    assert st["max_rel_residual"] <= 1e-7 and st["converged_cols"] == k, (name, st)
    assert np.all(np.isinf(R[network.floating_mask(inst)]))


def test_mg_cuts_iterations_and_is_deterministic(er):
    inst = I.precision_4x512(W=256, H=256, n_tsv=500, n_clusters=10)
    k, seed = 64, 9
    Rj, stj = run(er, inst, k, seed, 0)
    Rm, stm = run(er, inst, k, seed, 1)
    Rm2, _ = run(er, inst, k, seed, 1)
    np.testing.assert_array_equal(Rm, Rm2)
    print(f"Jacobi {stj['iterations']} iterations, multigrid {stm['iterations']}")
    assert stm["iterations"] * 5 <= stj["iterations"], (stj["iterations"], stm["iterations"])
    # both stop at the same accurate residual, so they agree to the accuracy that tol gives
    assert rel_err(Rm, Rj) <= 5e-4


def test_mg_option_rules(er):
    inst = I.tiny_plain()
    g = er.grid_create(inst)
    Y = torch.zeros((inst.n, 8), dtype=torch.float64, device="cuda")
    Z = torch.zeros_like(Y)
    with pytest.raises(er.ErError):
        er.solve(g, Y, Z, 8, "fp64", er.default_solve_opts("fp64", precond=1))
    with pytest.raises(er.ErError):
        er.solve(g, Y.float(), Z.float(), 8, "fp32", er.default_solve_opts("fp32", precond=2))
    R = [torch.empty(inst.n, dtype=torch.float64, device="cuda")] * 2
    with pytest.raises(er.ErError):  # no such preconditioner
        er.batch_solve([g], 8, 1, R[:1], opts=er.default_solve_opts("fp32", precond=2))
    with pytest.raises(er.ErError):  # the multigrid batch solves networks concurrently: no grid twice
        er.batch_solve([g, g], 8, 1, R, opts=er.default_solve_opts("fp32", precond=1))
    g.destroy()
