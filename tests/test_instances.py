"""The synthetic workloads match the recipes they stand for (CPU).

Each seeded generator in paper_2607_05818_gb300/instances.py stands in for a workload of
the paper's scale (its industrial benchmarks are not available).  These tests pin what the
recipes state: sizes, TSV and pad counts and values, the resistance distributions, the
share of open segments, and that a seed reproduces the same network.
"""
import numpy as np

from paper_2607_05818_gb300 import instances as I


def _seg_r(inst):
    gx, gy = inst.gx[inst.gx > 0], inst.gy[inst.gy > 0]
    return 1.0 / gx, 1.0 / gy


def test_tiny_plain_recipe():
    inst = I.tiny_plain()
    assert (inst.T, inst.W, inst.H, inst.n) == (2, 32, 32, 2048)
    assert len(inst.tsv_g) == 16 and np.allclose(1.0 / inst.tsv_g, 0.02)
    assert len({(x, y) for x, y in zip(inst.tsv_x, inst.tsv_y)}) == 16  # distinct positions
    assert len(inst.pad_g) == 16 and np.allclose(1.0 / inst.pad_g, 0.01)
    assert np.all(inst.pad_tier == 0) and np.all(inst.pad_x % 8 == 0) and np.all(inst.pad_y % 8 == 0)
    for t, base in enumerate((0.05, 0.10)):
        r = 1.0 / np.concatenate([inst.gx[t].ravel(), inst.gy[t].ravel()])
        assert abs(np.median(np.log(r / base))) < 0.02      # lognormal(0, 0.1) around base
        assert 0.09 < np.std(np.log(r)) < 0.11


def test_precision_recipe():
    inst = I.precision_4x512()
    assert (inst.T, inst.W, inst.H, inst.n) == (4, 512, 512, 1_048_576)
    assert len(inst.tsv_g) == 2000 * 3                      # 2,000 columns, one segment per tier pair
    r_t = 1.0 / inst.tsv_g
    assert r_t.min() >= 0.01 and r_t.max() <= 0.05
    cols = {(x, y) for x, y in zip(inst.tsv_x, inst.tsv_y)}
    assert len(cols) == 2000
    assert len(inst.pad_g) == 1024 and np.allclose(1.0 / inst.pad_g, 0.01)
    assert np.all(inst.gx > 0) and np.all(inst.gy > 0)      # no open segments
    for t in range(4):
        for g in (inst.gx[t], inst.gy[t]):
            lr = np.log(1.0 / g.ravel())
            assert np.log(0.02) - 0.05 < np.median(lr) < np.log(0.2) + 0.05   # log-uniform tier base
            assert 0.19 < np.std(lr) < 0.21                                    # lognormal(0.2) jitter
    # the 2 x 512^2 profiling case is the same recipe on half the tiers and TSVs
    half = I.precision_2x512()
    assert (half.T, half.W, half.H) == (2, 512, 512) and len(half.tsv_g) == 1000


def test_large_recipe():
    inst = I.large_8x1024()
    assert (inst.T, inst.W, inst.H, inst.n) == (8, 1024, 1024, 8_388_608)
    assert len(inst.tsv_g) == 20000 * 7
    assert len({(x, y) for x, y in zip(inst.tsv_x, inst.tsv_y)}) == 20000
    assert len(inst.pad_g) == 1024 and np.allclose(1.0 / inst.pad_g, 0.005)
    open_share = (np.sum(inst.gx == 0) + np.sum(inst.gy == 0)) / (inst.gx.size + inst.gy.size)
    assert abs(open_share - 0.10) < 0.002
    for t in range(8):
        base = 0.1 if t % 2 == 0 else 0.02
        r = 1.0 / inst.gx[t][inst.gx[t] > 0]
        assert abs(np.median(np.log(r / base))) < 0.01


def test_batch_recipe():
    cands = I.batch_candidates(64)
    for c in cands:
        assert c.T in (2, 3, 4) and c.W == c.H and c.W in (64, 128, 256)
        cols = len(c.tsv_g) // (c.T - 1)
        assert 50 <= cols <= 800 and len(c.tsv_g) == cols * (c.T - 1)
        assert len(c.pad_g) == (c.W // 16) ** 2
    assert len({(c.T, c.W) for c in cands}) >= 6              # the sizes really vary


def test_seeds_reproduce():
    a, b = I.precision_2x512(), I.precision_2x512()
    assert np.array_equal(a.gx, b.gx) and np.array_equal(a.tsv_x, b.tsv_x) and np.array_equal(a.tsv_g, b.tsv_g)
    c = I.precision_4x512(seed=I.BASE_SEED + 99, T=2, n_tsv=1000, n_clusters=20)
    assert not np.array_equal(a.gx, c.gx)
