"""Pins of the CPU oracle against closed forms, identities and brute force (no GPU).

Each test fixes the oracle to something other than itself: textbook networks,
Wu's closed form (Eq. 3), the paper's reduced TSV system (Eq. 10 and Eq. 13-15),
Foster's theorem, Rayleigh monotonicity, the Eq. 2 pseudo-inverse route, the
Eq. 4 Green's-function identity, Kirchhoff's current law, published SplitMix64
outputs and JL statistics.
"""
import json
import os

import numpy as np
import pytest

from oracle import exact, network, pairs, reduced, sketch, wu
from paper_2607_05818_gb300 import instances as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def nid(inst, t, x, y):
    return (t * inst.H + y) * inst.W + x


# ---------------------------------------------------------------- closed forms

def test_textbook_networks_golden():
    cases = json.load(open(os.path.join(GOLD, "textbook_networks.json")))["cases"]
    for c in cases:
        pads = c.get("pads", [c.get("pad")])
        inst = I.uniform(1, c["W"], c["H"], c["r"], c["s"],
                         pads=[(0, p[0], p[1], p[2]) for p in pads])
        R = exact.reff_dense(inst)
        for key, want in c["expect"].items():
            x, y = map(int, key.split(","))
            assert R[nid(inst, 0, x, y)] == pytest.approx(want, rel=1e-13), c["name"]


def test_P1_single_node_behind_pad():
    for r in (0.01, 0.5, 3.0):
        inst = I.uniform(1, 1, 1, 1.0, 1.0, pads=[(0, 0, 0, r)])
        assert exact.reff_dense(inst)[0] == pytest.approx(r, rel=1e-15)


def test_P2_series_chain_with_jitter():
    rng = np.random.default_rng(1)
    L = 17
    rx = rng.uniform(0.01, 0.3, (1, 1, L - 1))
    ry = np.zeros((1, 0, L))
    g = 37.0
    inst = I.from_resistances(rx, ry, pads=[(0, 0, 0, 1 / g)])
    R = exact.reff_dense(inst)
    want = 1 / g + np.concatenate([[0.0], np.cumsum(rx[0, 0])])
    np.testing.assert_allclose(R, want, rtol=1e-13)


def test_P3_parallel_tsvs_combine_harmonically():
    rt = [0.02, 0.05, 0.013, 0.04]
    g = 80.0
    inst = I.uniform(2, 1, 1, 1.0, 1.0, tsv=[(0, 0, 0, r) for r in rt], pads=[(0, 0, 0, 1 / g)])
    R = exact.reff_dense(inst)
    assert R[1] == pytest.approx(1 / g + 1 / sum(1 / r for r in rt), rel=1e-14)


def test_P5_wu_closed_form_single_tier():
    """Eq. 3: one uniform tier, one pad of conductance g at b: R_i = 1/g + R_Wu(b, i)."""
    for (M, N, r, s, b) in [(7, 5, 0.3, 0.7, (2, 3)), (9, 9, 0.05, 0.05, (0, 0)),
                            (12, 4, 0.2, 0.02, (11, 1)), (1, 6, 0.1, 0.4, (0, 2))]:
        g = 40.0
        inst = I.uniform(1, M, N, r, s, pads=[(0, b[0], b[1], 1 / g)])
        R = exact.reff_dense(inst)
        for y in range(N):
            for x in range(M):
                want = 1 / g + wu.reff_wu(M, N, r, s, b, (x, y))
                assert R[nid(inst, 0, x, y)] == pytest.approx(want, rel=1e-12)


def test_P5_multiple_angle_recursion_matches_cos():
    """Sec. III-E: the cosine table by recursion equals direct cos calls."""
    for M in (2, 5, 16, 33):
        np.testing.assert_allclose(np.asarray(wu.cos_half_table(M), float),
                                   np.asarray(wu.cos_half_direct(M), float), atol=1e-15)
    assert wu.reff_wu(9, 7, 0.3, 0.2, (1, 2), (7, 5), recursion=True) == pytest.approx(
        wu.reff_wu(9, 7, 0.3, 0.2, (1, 2), (7, 5)), rel=1e-14)


@pytest.mark.parametrize("d", [2, 3, 4])
def test_P6_paper_reduced_system_matches_full_network(d):
    """Eq. 6-10 and Eq. 13-15 on uniform stacks with through-stack TSVs: the bump-to-load
    resistance from the reduced TSV system equals the full-network Cholesky value."""
    rng = np.random.default_rng(10 + d)
    M, N = 6, 5
    rr = rng.uniform(0.1, 0.6, d)
    ss = rng.uniform(0.1, 0.6, d)
    p = 4
    pos = set()
    while len(pos) < p:
        pos.add((int(rng.integers(0, M)), int(rng.integers(0, N))))
    tsv = sorted(pos)
    Rt = rng.uniform(0.01, 0.08, (d - 1, p))
    st = reduced.UniformStack(M, N, rr, ss, tsv, Rt)
    bumps = [(3, 2), (0, 0)]
    loads = [(0, 4), (5, 1), (2, 2)]
    pairs = reduced.TransformedSystem(st).pairs(bumps, loads)
    tsvlist = [(t, x, y, Rt[t, k]) for k, (x, y) in enumerate(tsv) for t in range(d - 1)]
    gp = 1e3
    for i, b in enumerate(bumps):
        inst = I.uniform(d, M, N, rr, ss, tsv=tsvlist, pads=[(0, b[0], b[1], 1 / gp)])
        R = exact.reff_dense(inst)
        for j, l in enumerate(loads):
            full = R[nid(inst, d - 1, l[0], l[1])] - 1 / gp
            kkt, I_, V = reduced.pair_reff_kkt(st, b, l)
            assert kkt == pytest.approx(full, rel=1e-12)
            assert pairs[i, j] == pytest.approx(full, rel=1e-12)
            # Eq. 9: the TSV currents of every interface sum to the unit current
            np.testing.assert_allclose(I_.reshape(d - 1, p).sum(axis=1), 1.0, rtol=1e-12)


# ------------------------------------------------------------------ brute force

def test_P4_three_independent_inverse_routes():
    """Cholesky diag(G^-1), Gauss-Jordan and the Eq. 2 pseudo-inverse agree on tiny instances."""
    rng = np.random.default_rng(4)
    for _ in range(12):
        inst = I.random_small(rng)
        if inst.n > 64:
            continue
        a = exact.reff_dense(inst)
        b = exact.reff_gauss_jordan(inst)
        np.testing.assert_allclose(a, b, rtol=1e-12)
        if not np.any(np.isinf(a)):
            np.testing.assert_allclose(a, exact.reff_pinv(inst), rtol=1e-9)


def test_floating_nodes_brute_force():
    """Nodes with no path to a pad get +inf; the rest equal the pinv route on the kept graph."""
    rng = np.random.default_rng(5)
    seen = 0
    for _ in range(40):
        inst = I.random_small(rng, T=1, W=int(rng.integers(3, 7)), H=int(rng.integers(3, 7)),
                              open_frac=0.45, n_pads=1)
        fl = network.floating_mask(inst)
        # brute-force reachability: relax every conducting edge n times
        u, v, w, _, pu, pw, _ = network.edge_list(inst)
        reach = np.zeros(inst.n, bool)
        reach[pu] = True
        m = w > 0
        for _ in range(inst.n):
            np.logical_or.at(reach, v[m], reach[u[m]])
            np.logical_or.at(reach, u[m], reach[v[m]])
        np.testing.assert_array_equal(fl, ~reach)
        R = exact.reff_dense(inst)
        assert np.all(np.isinf(R[fl])) and np.all(np.isfinite(R[~fl]))
        seen += int(fl.any())
    assert seen > 0


def test_P7_foster_theorem():
    """sum_e w_e R_e = number of non-supply nodes (connected graph with the supply node)."""
    rng = np.random.default_rng(7)
    for _ in range(6):
        inst = I.random_small(rng)
        if np.any(network.floating_mask(inst)):
            continue
        Ginv, keep = exact.dense_inverse(inst)
        pos = {int(k): i for i, k in enumerate(keep)}
        u, v, w, _, pu, pw, _ = network.edge_list(inst)
        tot = 0.0
        for a, b, g in zip(u, v, w):
            ia, ib = pos[int(a)], pos[int(b)]
            tot += g * (Ginv[ia, ia] + Ginv[ib, ib] - 2 * Ginv[ia, ib])
        for a, g in zip(pu, pw):
            tot += g * Ginv[pos[int(a)], pos[int(a)]]
        assert tot == pytest.approx(inst.n, rel=1e-11)


def test_P8_rayleigh_monotonicity():
    """Raising a conductance (or adding a TSV) never increases any R_i."""
    rng = np.random.default_rng(8)
    for _ in range(8):
        inst = I.random_small(rng, T=2, W=5, H=4)
        R0 = exact.reff_dense(inst)
        up = I.Instance(**{**inst.__dict__})
        up.gx = inst.gx.copy()
        up.gx.flat[int(rng.integers(0, up.gx.size))] *= 3.0
        up.tsv_tier = np.append(inst.tsv_tier, 0).astype(np.int32)
        up.tsv_x = np.append(inst.tsv_x, 2).astype(np.int32)
        up.tsv_y = np.append(inst.tsv_y, 1).astype(np.int32)
        up.tsv_g = np.append(inst.tsv_g, 25.0)
        R1 = exact.reff_dense(up)
        assert np.all(R1 <= R0 * (1 + 1e-13))
        assert np.any(R1 < R0 * (1 - 1e-6))


def test_P9_scaling_and_mirror_symmetry():
    rng = np.random.default_rng(9)
    inst = I.random_small(rng, T=2, W=6, H=5)
    c = 3.7
    np.testing.assert_allclose(exact.reff_dense(inst.scaled(c)), c * exact.reff_dense(inst), rtol=1e-12)
    Rj, _ = sketch.reff_jl_dense(inst, 32, 11)
    Rjc, _ = sketch.reff_jl_dense(inst.scaled(c), 32, 11)
    np.testing.assert_allclose(Rjc, c * Rj, rtol=1e-12)
    # mirror-symmetric uniform instance -> mirror-symmetric R
    M, N = 7, 5
    sym = I.uniform(2, M, N, [0.1, 0.2], [0.3, 0.15],
                    tsv=[(0, 1, 2, 0.02), (0, 5, 2, 0.02)],
                    pads=[(0, 3, 0, 0.01), (0, 3, 4, 0.01)])
    R = exact.reff_dense(sym).reshape(2, N, M)
    np.testing.assert_allclose(R, R[:, :, ::-1], rtol=1e-12)
    np.testing.assert_allclose(R, R[:, ::-1, :], rtol=1e-12)


def test_P11_eq4_green_function_identity():
    """Eq. 4: with node b grounded, (G_b^-1)_{jk} = (R_bj + R_bk - R_jk) / 2 where R is the
    Eq. 2 pairwise resistance."""
    rng = np.random.default_rng(11)
    inst = I.random_small(rng, T=2, W=4, H=3, n_pads=1)
    L = network.laplacian_with_supply(inst)[:-1, :-1]
    # drop the pad terms: a pure mesh+TSV Laplacian
    L = L - np.diag(L.sum(axis=1))
    b = 0
    keep = [i for i in range(L.shape[0]) if i != b]
    Gb_inv = np.linalg.inv(L[np.ix_(keep, keep)])
    for jj, j in enumerate(keep[:5]):
        for kk, k in enumerate(keep[:5]):
            Rbj = exact.pair_reff_pinv(L, b, j)
            Rbk = exact.pair_reff_pinv(L, b, k)
            Rjk = exact.pair_reff_pinv(L, j, k) if j != k else 0.0
            assert Gb_inv[jj, kk] == pytest.approx(0.5 * (Rbj + Rbk - Rjk), rel=1e-9)


# ------------------------------------------------------- pairwise R and IR drop

def test_P12_pairs_and_drop_on_a_chain():
    """1 x L chain with one pad of resistance 1/g at x = 0: R(u, v) is the sum of the segments
    between u and v (the only path), and a current I drawn at x_l lowers node x by
    I (1/g + sum of the segments below min(x, x_l))."""
    rng = np.random.default_rng(41)
    L = 13
    rx = rng.uniform(0.01, 0.3, (1, 1, L - 1))
    g = 25.0
    inst = I.from_resistances(rx, np.zeros((1, 0, L)), pads=[(0, 0, 0, 1 / g)])
    cum = np.concatenate([[0.0], np.cumsum(rx[0, 0])])
    Rp = pairs.pair_reff_exact(inst, np.arange(L), np.arange(L))
    np.testing.assert_allclose(Rp, np.abs(cum[:, None] - cum[None, :]), rtol=1e-12, atol=1e-14)
    loads = [4, 9]
    cur = np.array([[2.0, 0.5], [1.0, -0.25]])  # two load scenarios
    drop = pairs.ir_drop_exact(inst, loads, cur)
    x = np.arange(L)
    for s in range(2):
        want = sum(cur[j, s] * (1 / g + cum[np.minimum(x, xl)]) for j, xl in enumerate(loads))
        np.testing.assert_allclose(drop[:, s], want, rtol=1e-12)


def test_P13_pair_reff_is_eq2_on_the_laplacian_with_supply():
    """Eq. 2 taken literally on the (n+1)-node Laplacian, paths through the supply included."""
    rng = np.random.default_rng(42)
    for _ in range(3):
        inst = I.random_small(rng, T=2, W=3, H=3, n_pads=2)
        L = network.laplacian_with_supply(inst)
        us, vs = rng.permutation(inst.n)[:4], rng.permutation(inst.n)[:5]
        Rp = pairs.pair_reff_exact(inst, us, vs)
        for a, u in enumerate(us):
            for b, v in enumerate(vs):
                want = 0.0 if u == v else exact.pair_reff_pinv(L, int(u), int(v))
                assert Rp[a, b] == pytest.approx(want, rel=1e-10, abs=1e-14)


def test_P14_drop_obeys_kcl_superposition_and_eq4():
    """G drop = I at every node (Kirchhoff's current law); drops of several loads add; and for a
    unit current at l, drop_i = (G^-1)_il = (R_i + R_l - R(i, l)) / 2 (Eq. 4 with the supply as
    the grounded node), from the map and the Eq. 2 pairwise resistance."""
    rng = np.random.default_rng(43)
    inst = I.random_small(rng, T=3, W=5, H=4, n_tsv=6, n_pads=2)
    loads = rng.choice(inst.n, 7, replace=False)
    cur = rng.uniform(-1.0, 2.0, (7, 3))
    drop = pairs.ir_drop_exact(inst, loads, cur)
    G = network.conductance_matrix(inst, dense=True)
    b = np.zeros((inst.n, 3))
    b[loads] = cur
    np.testing.assert_allclose(G @ drop, b, rtol=0, atol=1e-10)
    parts = sum(pairs.ir_drop_exact(inst, [l], cur[j:j + 1]) for j, l in enumerate(loads))
    np.testing.assert_allclose(parts, drop, rtol=1e-11)
    Rs = exact.reff_dense(inst)
    Lp = network.laplacian_with_supply(inst)
    l = int(loads[0])
    unit = pairs.ir_drop_exact(inst, [l], [1.0])[:, 0]
    for i in range(inst.n):
        Ril = 0.0 if i == l else exact.pair_reff_pinv(Lp, i, l)
        assert unit[i] == pytest.approx(0.5 * (Rs[i] + Rs[l] - Ril), rel=1e-9)


def test_P15_jl_pairs_and_drop_statistics_and_same_seed_identities():
    """Over seeds the JL pair and drop estimates average to the exact values; for one seed,
    R_JL(u, v) = R_JL,u + R_JL,v - 2 drop_JL(u; unit current at v) and drop_JL(u; unit at u) =
    R_JL,u, tying both to the R map of the same sketch."""
    rng = np.random.default_rng(44)
    inst = I.random_small(rng, T=2, W=4, H=3, n_tsv=3, n_pads=2)
    us, vs = np.array([0, 5, 13, 22]), np.array([1, 7, 13, 20, 23])
    loads, cur = np.array([3, 17, 22]), np.array([1.0, 0.5, 2.0])
    Rex = pairs.pair_reff_exact(inst, us, vs)
    Dex = pairs.ir_drop_exact(inst, loads, cur)[:, 0]
    fl = network.floating_mask(inst)
    k, S = 32, 256
    Rs, Ds = [], []
    for s in range(S):
        Rmap, Z = sketch.reff_jl_dense(inst, k, 900 + s)
        Rs.append(pairs.pair_reff_jl(Z, fl, us, vs))
        Ds.append(pairs.ir_drop_jl(Z, fl, loads, cur)[:, 0])
        if s == 0:
            for a, u in enumerate(us):
                for b, v in enumerate(vs):
                    unit_v = pairs.ir_drop_jl(Z, fl, [v], [1.0])[u, 0]
                    assert Rs[0][a, b] == pytest.approx(Rmap[u] + Rmap[v] - 2 * unit_v, rel=1e-10, abs=1e-13)
            for u in us:
                assert pairs.ir_drop_jl(Z, fl, [u], [1.0])[u, 0] == pytest.approx(Rmap[u], rel=1e-12)
    Rs, Ds = np.stack(Rs), np.stack(Ds)
    off = us[:, None] != vs[None, :]
    assert np.all(Rs[:, ~off] == 0.0)
    assert np.all(np.abs(Rs.mean(0) - Rex)[off] <= 4 * (Rs.std(0) / np.sqrt(S))[off])
    assert np.all(np.abs(Ds.mean(0) - Dex) <= 4 * Ds.std(0) / np.sqrt(S) + 1e-15)


def test_pairs_and_drop_with_floating_nodes():
    """Pairs touching a floating node and drops at one are +inf; currents at floating nodes are
    ignored (no path to the supply); the rest equals the network without those currents."""
    rng = np.random.default_rng(45)
    for _ in range(20):
        inst = I.random_small(rng, T=1, W=6, H=5, n_pads=1, open_frac=0.4)
        fl = network.floating_mask(inst)
        if fl.any() and (~fl).sum() >= 3:
            break
    assert fl.any()
    us, vs = np.arange(inst.n), np.arange(inst.n)
    Rp = pairs.pair_reff_exact(inst, us, vs)
    assert np.all(np.isinf(Rp[fl, :])) and np.all(np.isinf(Rp[:, fl]))
    assert np.all(np.isfinite(Rp[np.ix_(~fl, ~fl)]))
    good, bad = np.flatnonzero(~fl)[:2], np.flatnonzero(fl)[:1]
    drop = pairs.ir_drop_exact(inst, np.concatenate([good, bad]), [1.0, 2.0, 5.0])[:, 0]
    ref = pairs.ir_drop_exact(inst, good, [1.0, 2.0])[:, 0]
    assert np.all(np.isinf(drop[fl]))
    np.testing.assert_allclose(drop[~fl], ref[~fl], rtol=1e-13)
    _, Z = sketch.reff_jl_dense(inst, 16, 3)
    dj = pairs.ir_drop_jl(Z, fl, np.concatenate([good, bad]), [1.0, 2.0, 5.0])[:, 0]
    assert np.all(np.isinf(dj[fl])) and np.all(np.isfinite(dj[~fl]))


def test_P16_pad_currents_obey_kcl_and_divide_by_conductance():
    """Pad currents add up to the load current (KCL with the supply); on a 1 x L chain with a
    pad at each end the current of a load at x splits in inverse proportion to the two
    resistances to the supply; the share statistic counts pads largest first."""
    rng = np.random.default_rng(46)
    inst = I.random_small(rng, T=2, W=6, H=5, n_tsv=5, n_pads=4)
    loads = rng.choice(inst.n, 6, replace=False)
    cur = rng.uniform(0.1, 1.0, (6, 2))
    pc = pairs.pad_currents(inst, pairs.ir_drop_exact(inst, loads, cur))
    np.testing.assert_allclose(pc.sum(axis=0), cur.sum(axis=0), rtol=1e-11)
    L, r, g1, g2, x = 9, 0.1, 20.0, 50.0, 3
    inst = I.from_resistances(np.full((1, 1, L - 1), r), np.zeros((1, 0, L)),
                              pads=[(0, 0, 0, 1 / g1), (0, L - 1, 0, 1 / g2)])
    pc = pairs.pad_currents(inst, pairs.ir_drop_exact(inst, [x], [1.0]))[:, 0]
    left, right = 1 / g1 + x * r, 1 / g2 + (L - 1 - x) * r
    np.testing.assert_allclose(pc, [right / (left + right), left / (left + right)], rtol=1e-12)
    assert pairs.bumps_for_share([5.0, 1.0, 1.0, 1.0, 2.0], 0.95) == 1.0
    assert pairs.bumps_for_share([90.0, 5.0, 3.0, 2.0], 0.95) == 0.5
    assert pairs.bumps_for_share([100.0, 0.0, 0.0, 0.0], 0.95) == 0.25


# --------------------------------------------------------------------- sketch

def test_splitmix64_published_stream():
    vals = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64_seed0.txt")) if l.startswith("0x")]
    gamma = np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        z = np.arange(len(vals), dtype=np.uint64) * gamma
    got = [int(v) for v in sketch.splitmix64(z)]
    assert got == vals


def test_sketch_c_matches_numpy(oracle_c_built):
    rng = np.random.default_rng(12)
    for _ in range(4):
        inst = I.random_small(rng, open_frac=0.2)
        for k in (1, 3, 32):
            np.testing.assert_allclose(sketch.sketch_c(inst, k, 99), sketch.sketch_numpy(inst, k, 99),
                                       rtol=0, atol=1e-14)


def test_sketch_rows_match_full_sketch():
    """Sampled rows (a per-node gather over incident edges) equal the full sketch's rows (an
    edge-major scatter), floating nodes and nodes with pads and TSVs included."""
    rng = np.random.default_rng(31)
    for _ in range(4):
        inst = I.random_small(rng, open_frac=0.25)
        Y = sketch.sketch_numpy(inst, 8, 17)
        nodes = rng.permutation(inst.n)[: max(1, inst.n // 2)]
        np.testing.assert_allclose(sketch.sketch_rows(inst, nodes, 8, 17), Y[nodes], rtol=0, atol=1e-14)
    with pytest.raises(ValueError):
        sketch.sketch_rows(inst, [0, 0], 8, 17)


def test_sketch_structure():
    """Mesh rows of M sum to zero over nodes, so the column sums of Y^T are the pad terms alone;
    entries are sums of +-sqrt(w/k) with the canonical sign convention."""
    inst = I.tiny_plain()
    k, seed = 16, 5
    Yt = sketch.sketch_numpy(inst, k, seed)
    _, _, _, _, pu, pw, peid = network.edge_list(inst)
    pad_part = (sketch.rademacher(seed, peid, k) * np.sqrt(pw / k)[:, None]).sum(axis=0)
    np.testing.assert_allclose(Yt.sum(axis=0), pad_part, atol=1e-12)
    # a single x-segment network: node 0 gets +sqrt(w/k) q, node 1 gets -sqrt(w/k) q
    one = I.uniform(1, 2, 1, 0.25, 1.0, pads=[(0, 0, 0, 1.0)])
    Y1 = sketch.sketch_numpy(one, 4, 3)
    q = sketch.rademacher(3, [0], 4)[0]
    np.testing.assert_allclose(Y1[1], -np.sqrt(4.0 / 4) * q, rtol=1e-15)


def test_sketch_second_moment_is_G():
    """E[Y^T Y] = M^T E[Q^T Q] M = G.  Over S seeds each entry's error has standard deviation
    sqrt(sum_{e<f} (M_ea M_fb + M_fa M_eb)^2 / k / S); every entry stays within 5 of them."""
    inst = I.random_small(np.random.default_rng(13), T=1, W=3, H=2, n_pads=1)
    G = network.conductance_matrix(inst, dense=True)
    n = inst.n
    u, v, w, _, pu, pw, _ = network.edge_list(inst)
    rows = []
    for a, b, g in zip(u, v, w):
        r = np.zeros(n)
        r[a], r[b] = np.sqrt(g), -np.sqrt(g)
        rows.append(r)
    for a, g in zip(pu, pw):
        r = np.zeros(n)
        r[a] = np.sqrt(g)
        rows.append(r)
    Mm = np.array(rows)
    np.testing.assert_allclose(Mm.T @ Mm, G, rtol=1e-13, atol=1e-12)
    k, S = 64, 200
    acc = np.zeros_like(G)
    for s in range(S):
        Y = sketch.sketch_numpy(inst, k, 1000 + s)
        acc += Y @ Y.T
    acc /= S
    var = np.zeros_like(G)
    m = Mm.shape[0]
    for e in range(m):
        for f in range(e + 1, m):
            c = np.outer(Mm[e], Mm[f]) + np.outer(Mm[f], Mm[e])
            var += c * c
    sd = np.sqrt(var / k / S)
    assert np.all(np.abs(acc - G) <= 5 * sd + 1e-9)


def test_P10_jl_statistics():
    """Mean of R_JL over seeds -> exact R; per-node relative spread about sqrt(2/k)."""
    inst = I.random_small(np.random.default_rng(14), T=2, W=4, H=4, n_pads=2)
    Rex = exact.reff_dense(inst)
    k = 32
    S = 256
    samples = np.stack([sketch.reff_jl_dense(inst, k, 500 + s)[0] for s in range(S)])
    mean = samples.mean(axis=0)
    sd = samples.std(axis=0)
    assert np.all(np.abs(mean - Rex) <= 3.5 * sd / np.sqrt(S) + 1e-15)
    rel_sd = sd / Rex
    assert np.all(rel_sd <= np.sqrt(2 / k) * 1.3)
    assert np.median(rel_sd) > 0.5 * np.sqrt(2 / k)


def test_jl_dense_matches_sparse_sampled():
    inst = I.tiny_plain()
    k, seed = 16, 3
    Yt = sketch.sketch_numpy(inst, k, seed)
    R, Z = sketch.reff_jl_dense(inst, k, seed, Yt)
    f = exact.SparseFactor(inst)
    nodes = [0, 5, 777, 2047]
    Rs, Zs = sketch.reff_jl_sampled(f, Yt, nodes)
    np.testing.assert_allclose(Rs, R[nodes], rtol=1e-12)
    np.testing.assert_allclose(Zs, Z[nodes], rtol=1e-10, atol=1e-14)
    Rex = exact.reff_dense(inst)
    np.testing.assert_allclose([f.reff(i) for i in nodes], Rex[nodes], rtol=1e-12)


def test_jl_with_floating_nodes_matches_sampled():
    """Floating nodes (no path to a pad) are excluded from the JL route too: R = +inf there
    and the kept rows equal exact sparse solves."""
    inst = I.random_small(np.random.default_rng(3), T=1, W=20, H=19, n_pads=1, open_frac=0.35)
    fl = network.floating_mask(inst)
    assert fl.any()
    k, seed = 8, 2
    Yt = sketch.sketch_numpy(inst, k, seed)
    R, Z = sketch.reff_jl_dense(inst, k, seed, Yt)
    assert np.all(np.isinf(R[fl])) and np.all(np.isfinite(R[~fl]))
    f = exact.SparseFactor(inst)
    nodes = np.flatnonzero(~fl)[:6]
    Rs, _ = sketch.reff_jl_sampled(f, Yt, nodes)
    np.testing.assert_allclose(R[nodes], Rs, rtol=1e-12)


# ------------------------------------------------------------------ U-Net reference

def test_unet_reference_gradient_matches_finite_differences():
    """The FP64 U-Net reference's backward pass against central finite differences on a tiny
    network (2 levels, 2 base channels, 4x4 maps): every parameter."""
    from oracle.unet_ref import UNetRef
    net = UNetRef(in_ch=3, out_ch=2, levels=2, base=2)
    rng = np.random.default_rng(21)
    flat = rng.normal(0, 0.5, net.num_params())
    x = rng.normal(0, 1, (2, 4, 4, 3))
    target = rng.normal(0, 1, (2, 4, 4, 2))
    mask = rng.random((2, 4, 4, 2)) > 0.2
    loss, grad, _ = net.loss_and_grad(flat, x, target, mask)
    h = 1e-6
    fd = np.zeros_like(flat)
    for i in range(len(flat)):
        e = np.zeros_like(flat)
        e[i] = h
        fd[i] = (net.loss_and_grad(flat + e, x, target, mask)[0] - net.loss_and_grad(flat - e, x, target, mask)[0]) / (2 * h)
    np.testing.assert_allclose(grad, fd, rtol=1e-5, atol=1e-8)


def test_unet_reference_layers_against_definitions():
    """conv3x3 against a direct loop; max pooling against a loop; upsampling round trip."""
    from oracle import unet_ref as U
    rng = np.random.default_rng(22)
    x = rng.normal(size=(1, 5, 4, 3))
    w = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    y = U.conv3x3(x, w, b)
    for (h, ww, o) in [(0, 0, 0), (4, 3, 1), (2, 1, 0)]:
        s = b[o]
        for ky in range(3):
            for kx in range(3):
                yy, xx = h + ky - 1, ww + kx - 1
                if 0 <= yy < 5 and 0 <= xx < 4:
                    s += x[0, yy, xx, :] @ w[o, ky, kx, :]
        assert y[0, h, ww, o] == pytest.approx(s, rel=1e-12)
    z = rng.normal(size=(1, 4, 4, 2))
    m, _ = U.maxpool(z)
    assert m[0, 1, 0, 1] == max(z[0, 2, 0, 1], z[0, 2, 1, 1], z[0, 3, 0, 1], z[0, 3, 1, 1])
    np.testing.assert_allclose(U.upsample_bwd(U.upsample(z)), 4 * z)
