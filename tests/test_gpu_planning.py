"""Through-bump currents and the TSV-planning sweep through the C ABI, against the oracle.

er_pad_currents on the GPU's exact IR drop (er_solve with the load currents as right-hand
sides) must match the oracle's g_pad * (G^-1 I) at the pads within the solve tolerance,
and add up to the load current (Kirchhoff's current law).  The sweep driver on small
band-like and uniform plans must give the oracle's bump-share statistic (to one bump, the
resolution of the count) and the paper's qualitative finding: a band concentrates the
current on fewer bumps than a uniform plan.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import pairs
from paper_2607_05818_gb300 import instances as I


@pytest.fixture(scope="module")
def er():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_05818_gb300 import er as mod
    return mod


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 1e-5)])
def test_pad_currents_match_oracle(er, prec, tol):
    inst = I.random_small(np.random.default_rng(21), T=3, W=37, H=23, n_tsv=40, n_pads=7)
    rng = np.random.default_rng(22)
    loads = rng.choice(np.arange(2 * inst.W * inst.H, inst.n), 60, replace=False)
    cur = rng.uniform(0.0, 0.1, (60, 4))
    B = np.zeros((inst.n, 4))
    np.add.at(B, loads, cur)
    dt = torch.float64 if prec == "fp64" else torch.float32
    g = er.grid_create(inst)
    Bd = torch.from_numpy(B).to("cuda", dt)
    V = torch.empty_like(Bd)
    opts = er.default_solve_opts(prec, tol=1e-13 if prec == "fp64" else 1e-8)
    er.solve(g, Bd, V, 4, prec, opts)
    Ip = torch.full((len(inst.pad_g), 4), float("nan"), dtype=torch.float64, device="cuda")
    er.pad_currents(g, V, 4, prec, Ip)
    torch.cuda.synchronize()
    got = Ip.cpu().numpy()
    ref = pairs.pad_currents(inst, pairs.ir_drop_exact(inst, loads, cur))
    tot = cur.sum(axis=0)
    assert np.all(np.abs(got - ref) <= tol * tot[None, :])
    np.testing.assert_allclose(got.sum(axis=0), tot, rtol=10 * tol)
    g.destroy()


def test_planning_sweep_small(er):
    from paper_2607_05818_gb300 import planning as P
    plans = [P.floorplan("band", n_tsv=64, W=64, H=64, band_rows=8),
             P.floorplan("uniform", n_tsv=64, W=64, H=64)]
    res, _ = P.sweep(plans, k=16)
    n_pads = len(plans[0].pad_g)
    for p, r in zip(plans, res):
        assert abs(r["pad_current_sum"] - r["load_current"]) <= 1e-5 * r["load_current"]
        loads, cur = P.block_loads(p)
        ref = pairs.bumps_for_share(pairs.pad_currents(p, pairs.ir_drop_exact(p, loads, cur)).sum(axis=1))
        assert abs(r["bump_share_95"] - ref) <= 1.0 / n_pads + 1e-12
        assert np.isfinite(r["max_R_at_loads"]) and r["max_R_at_loads"] > 0
    assert res[0]["bump_share_95"] < res[1]["bump_share_95"]
