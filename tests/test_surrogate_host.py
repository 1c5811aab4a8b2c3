"""Host logic of the surrogate (CPU): the per-node input maps, the targets, the BF16
rounding used to upload them and the screening score, against their stated definitions."""
import numpy as np

from paper_2607_05818_gb300 import instances as I
from paper_2607_05818_gb300 import surrogate as S


def test_node_maps_encode_each_tier():
    inst = I.random_small(np.random.default_rng(5), T=3, W=9, H=7, n_tsv=6, n_pads=2)
    m = S.node_maps(inst)
    assert m.shape == (7, 9, 32) and m.dtype == np.float32
    enc = lambda g: np.log1p(g) / 4.0  # noqa: E731  ln(1 + g) / 4, 0 where absent
    for t in range(3):
        np.testing.assert_allclose(m[:, :8, 4 * t], enc(inst.gx[t]), rtol=1e-6)
        np.testing.assert_allclose(m[:6, :, 4 * t + 1], enc(inst.gy[t]), rtol=1e-6)
        assert np.all(m[:, 8, 4 * t] == 0) and np.all(m[6, :, 4 * t + 1] == 0)
    tsv = np.zeros((3, 7, 9))
    for tier, x, y, g in zip(inst.tsv_tier, inst.tsv_x, inst.tsv_y, inst.tsv_g):
        tsv[tier, y, x] += g        # a TSV segment touches both of its tiers
        tsv[tier + 1, y, x] += g
    pad = np.zeros((3, 7, 9))
    for tier, x, y, g in zip(inst.pad_tier, inst.pad_x, inst.pad_y, inst.pad_g):
        pad[tier, y, x] += g
    for t in range(3):
        np.testing.assert_allclose(m[:, :, 4 * t + 2], enc(tsv[t]), rtol=1e-5)
        np.testing.assert_allclose(m[:, :, 4 * t + 3], enc(pad[t]), rtol=1e-5)
    assert np.all(m[:, :, 12:] == 0)  # channel padding to a multiple of 32


def test_target_map_masks_infinite():
    inst = I.random_small(np.random.default_rng(6), T=2, W=4, H=3, n_pads=1)
    R = np.arange(1, inst.n + 1, dtype=np.float64)
    R[5] = np.inf
    t, m = S.target_map(R, inst)
    assert t.shape == (3, 4, 2) and m.shape == (3, 4, 2)
    tier, rem = divmod(5, 12)
    y, x = divmod(rem, 4)
    assert m[y, x, tier] == 0 and t[y, x, tier] == 0 and m.sum() == inst.n - 1
    assert np.isclose(t[0, 1, 1], np.log(R[12 + 1]))


def test_bf16_round_to_nearest_even():
    a = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-5, 65504.0], dtype=np.float32)
    b = S.bf16_bits(a)
    back = (b.astype(np.uint32) << 16).view(np.float32)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: even mantissa (1) wins; 1 + 3*2^-8 rounds up
    np.testing.assert_array_equal(back[:3], np.array([1.0, 1.0, 1.0 + 2 ** -6], dtype=np.float32))
    assert back[3] == -2.5
    assert np.all(np.abs(back[4:] / a[4:] - 1) <= 2 ** -8)


def test_score_is_the_99th_percentile_of_finite_nodes():
    v = np.arange(1000, dtype=np.float64).reshape(10, 10, 10)
    mask = np.ones_like(v, dtype=np.uint8)
    mask.ravel()[-5:] = 0  # the five largest are not finite nodes
    assert S.score(v, mask) == np.percentile(np.arange(995), 99)
    assert S.score(v) == np.percentile(np.arange(1000), 99)
