"""Host logic of the TSV-planning sweep (CPU): the plans it draws and the statistic it reads
off the through-bump currents (Sec. IV-B), against the oracle's definition."""
import numpy as np
import pytest

from oracle import pairs
from paper_2607_05818_gb300 import planning as PL


@pytest.mark.parametrize("seed", range(6))
def test_bump_share_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    for n in (1, 2, 7, 64, 1024):
        c = rng.lognormal(0.0, 2.0, n) * rng.choice([-1.0, 1.0], n)  # signs: magnitudes count
        c[rng.random(n) < 0.1] = 0.0
        assert PL.bump_share(c) == pytest.approx(pairs.bumps_for_share(c), abs=1e-12)
        c2 = np.round(np.abs(c), 1)  # ties
        assert PL.bump_share(c2) == pytest.approx(pairs.bumps_for_share(c2), abs=1e-12)


@pytest.mark.parametrize("pattern,count,rows", [("band", 1024, 32), ("band", 512, 64), ("uniform", 2048, 32)])
def test_tsv_plans(pattern, count, rows):
    W = H = 256
    xs, ys = PL.tsv_plan(W, H, count, pattern, rows)
    assert len(xs) == count and len(set(zip(xs.tolist(), ys.tolist()))) == count  # distinct columns
    assert xs.min() >= 0 and xs.max() < W and ys.min() >= 0 and ys.max() < H
    if pattern == "band":
        y0 = (H - rows) // 2
        assert ys.min() >= y0 and ys.max() < y0 + rows
    else:
        assert ys.max() - ys.min() > H // 2  # spread over the die


def test_blocks_and_loads():
    inst = PL.floorplan("band", n_tsv=256, T=2, W=64, H=64, r_tier=(0.05, 0.1))
    bl = PL.blocks(64, 64)
    assert len(bl) == 4
    for x0, y0, bw, bh in bl:
        assert 0 <= x0 and x0 + bw <= 64 and 0 <= y0 and y0 + bh <= 64 and bw == 2 * bh
    loads, cur = PL.block_loads(inst)
    top = (inst.T - 1) * inst.W * inst.H
    assert loads.min() >= top and loads.max() < inst.n
    np.testing.assert_allclose(cur.sum(axis=0), 1.0)  # one ampere per block scenario
    assert np.all((cur > 0).sum(axis=1) == 1)          # each load node belongs to one block
