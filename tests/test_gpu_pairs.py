"""Pairwise effective resistance and IR drop from Z through the C ABI, against the oracle.

Two layers: (1) the kernels alone, fed the oracle's own same-seed Z (uploaded), must
reproduce the oracle's ||Z_u - Z_v||^2 and Z (Z^T I) to FP64 rounding; (2) the whole path
(GPU sketch + solve + pair/drop kernels) against the oracle's same-seed values, within
1e-9 (FP64) or 1e-3 (FP32 form) of the natural scale of each quantity: R_u + R_v for a
pair (the size of the terms that cancel in Eq. 4) and ||Z_i|| ||w|| for a drop (the
Cauchy-Schwarz bound of the dot product).  Sizes span several 64 x 64 pair tiles with
ragged edges, ragged k, floating nodes, repeated ids and several load scenarios.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import network, pairs
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


def _pair_and_drop(er, g, Z, k, prec, us, vs, loads, cur):
    n = Z.shape[0]
    Rp = torch.full((len(us), len(vs)), float("nan"), dtype=torch.float64, device=DEV)
    S = 1 if np.ndim(cur) == 1 else np.shape(cur)[1]
    D = torch.full((n, S), float("nan"), dtype=torch.float64, device=DEV)
    er.pair_reff(g, Z, k, prec, us, vs, Rp)
    er.ir_drop(g, Z, k, prec, loads, cur, D)
    torch.cuda.synchronize()
    return Rp.cpu().numpy(), D.cpu().numpy()


def _check_pairs(got, ref, Rmap, us, vs, tol):
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    scale = (Rmap[us][:, None] + Rmap[vs][None, :])[fin]
    assert np.all(np.abs(got[fin] - ref[fin]) <= tol * scale)


def _check_drop(got, ref, Z, loads, cur, fl, tol):
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    b = np.zeros((Z.shape[0], ref.shape[1]))
    np.add.at(b, loads, np.asarray(cur).reshape(len(loads), -1))
    w = Z.T @ b
    scale = np.linalg.norm(Z, axis=1)[:, None] * np.linalg.norm(w, axis=0)[None, :] + 1e-300
    assert np.all(np.abs(got - ref)[fin] <= tol * scale[fin])


CASES = [
    # name, instance, k, m, nv, loads, scenarios
    ("tiny_plain_k128", lambda: I.tiny_plain(), 128, 70, 133, 50, 3),
    ("ragged_3x37x23_k36", lambda: I.random_small(np.random.default_rng(1), T=3, W=37, H=23, n_tsv=40, n_pads=3),
     36, 65, 129, 300, 1),
    ("floating_1x20x19_k20", lambda: I.random_small(np.random.default_rng(3), T=1, W=20, H=19, n_pads=1,
                                                    open_frac=0.35), 20, 64, 64, 40, 8),
]


@pytest.mark.parametrize("name,make,k,m,nv,nl,S", CASES, ids=[c[0] for c in CASES])
def test_kernels_on_the_oracle_Z(er, name, make, k, m, nv, nl, S):
    """The pair and drop kernels alone: the oracle's same-seed Z uploaded, both precisions."""
    inst = make()
    rng = np.random.default_rng(7)
    us = rng.integers(0, inst.n, m)
    vs = rng.integers(0, inst.n, nv)
    vs[:3] = us[:3]  # u == v pairs
    loads = rng.integers(0, inst.n, nl)
    cur = rng.uniform(-0.5, 2.0, (nl, S))
    _, Zo = osk.reff_jl_dense(inst, k, 99)
    fl = network.floating_mask(inst)
    g = er.grid_create(inst)
    for prec, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        Zin = Zo.astype(np.float32).astype(np.float64) if prec == "fp32" else Zo
        Zd = torch.from_numpy(Zin).to(DEV, dt).contiguous()
        Rp, D = _pair_and_drop(er, g, Zd, k, prec, us, vs, loads, cur)
        Rref = pairs.pair_reff_jl(Zin, fl, us, vs)
        Dref = pairs.ir_drop_jl(Zin, fl, loads, cur)
        Rmap = np.sum(Zin * Zin, axis=1)
        # FP64: rounding only; FP32 inputs: FP32 differences and partial sums
        tol = 1e-13 if prec == "fp64" else 1e-5
        _check_pairs(Rp, Rref, Rmap, us, vs, tol)
        assert np.all(Rp[np.arange(3), np.arange(3)][~fl[us[:3]]] == 0.0)
        _check_drop(D, Dref, Zin, loads, cur, fl, tol)
    g.destroy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 1e-3)])
def test_whole_path_against_oracle(er, prec, tol):
    """GPU sketch + solve + pair/drop kernels against the oracle's same-seed estimates."""
    inst = I.tiny_plain()
    k, seed = 128, 20260701
    dt = torch.float64 if prec == "fp64" else torch.float32
    g = er.grid_create(inst)
    Yt = torch.empty((inst.n, k), dtype=dt, device=DEV)
    Z = torch.empty_like(Yt)
    er.sketch(g, k, seed, prec, Yt)
    er.solve(g, Yt, Z, k, prec)
    pads = np.flatnonzero(np.isin(np.arange(inst.n), network.node_id(inst.T, inst.W, inst.H, inst.pad_tier,
                                                                        inst.pad_y, inst.pad_x)))
    top = np.arange((inst.T - 1) * inst.W * inst.H, inst.n)
    rng = np.random.default_rng(8)
    loads = rng.choice(top, 200, replace=False)
    cur = rng.uniform(0.0, 1e-3, (200, 2))
    Rp, D = _pair_and_drop(er, g, Z, k, prec, pads, top, loads, cur)
    Rmap, Zo = osk.reff_jl_dense(inst, k, seed)
    fl = network.floating_mask(inst)
    _check_pairs(Rp, pairs.pair_reff_jl(Zo, fl, pads, top), Rmap, pads, top, tol)
    _check_drop(D, pairs.ir_drop_jl(Zo, fl, loads, cur), Zo, loads, cur, fl, tol)
    g.destroy()


def test_invalid_arguments(er):
    inst = I.tiny_plain()
    g = er.grid_create(inst)
    Z = torch.zeros((inst.n, 8), dtype=torch.float64, device=DEV)
    R = torch.zeros((2, 2), dtype=torch.float64, device=DEV)
    with pytest.raises(er.ErError):
        er.pair_reff(g, Z, 8, "fp64", [0, inst.n], [1, 2], R)
    with pytest.raises(er.ErError):
        er.pair_reff(g, Z, 8, "fp64", [0, -1], [1, 2], R)
    D = torch.zeros((inst.n, 9), dtype=torch.float64, device=DEV)
    with pytest.raises(er.ErError):
        er.ir_drop(g, Z, 8, "fp64", [0], np.ones((1, 9)), D)  # S > 8
    with pytest.raises(er.ErError):
        er.ir_drop(g, Z, 8, "fp64", [0], [np.nan], D)
    # empty pair sets are a no-op; no loads gives a zero drop
    er.pair_reff(g, Z, 8, "fp64", [], [1, 2], R)
    D1 = torch.full((inst.n, 1), 7.0, dtype=torch.float64, device=DEV)
    er.ir_drop(g, Z, 8, "fp64", np.zeros(0, np.int64), np.zeros(0), D1)
    torch.cuda.synchronize()
    assert float(D1.abs().max()) == 0.0
    g.destroy()
