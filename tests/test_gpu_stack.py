"""The paper's own pipeline (Wu's closed form, the reduced TSV system of Eq. 13, one LU,
m + n solves, Eq. 15 pair dots) through the C ABI, against the oracle's reduced-system
implementation (long-double Wu sums, LAPACK LU), which the CPU pins tie to full Cholesky
solves of the same stack.  Sizes span several 32-column LU panels with a ragged last
panel, several 16 x 64 pair-dot tiles with ragged edges, d = 2 (bump and load blocks
coincide), duplicated bump positions and a bump sitting on a TSV.
"""
import zlib

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import reduced


@pytest.fixture(scope="module")
def er():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_05818_gb300 import er as mod
    return mod


def make_stack(rng, M, N, d, p, m, n):
    r = rng.uniform(0.02, 0.2, d)
    s = rng.uniform(0.02, 0.2, d)
    cells = rng.choice(M * N, p, replace=False)
    tsv = np.stack([cells % M, cells // M], axis=1)
    Rt = rng.uniform(0.01, 0.05, (d - 1, p))
    bumps = np.stack([rng.integers(0, M, m), rng.integers(0, N, m)], axis=1)
    loads = np.stack([rng.integers(0, M, n), rng.integers(0, N, n)], axis=1)
    return r, s, tsv, Rt, bumps, loads


CASES = [
    ("d2_12x9_p5", 12, 9, 2, 5, 3, 7),
    ("d3_16x16_p12", 16, 16, 3, 12, 5, 70),
    ("d4_24x20_p33", 24, 20, 4, 33, 17, 65),
    ("d5_7x31_p9", 7, 31, 5, 9, 2, 3),
]


@pytest.mark.parametrize("name,M,N,d,p,m,n", CASES, ids=[c[0] for c in CASES])
def test_stack_pairs_match_oracle(er, name, M, N, d, p, m, n):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    r, s, tsv, Rt, bumps, loads = make_stack(rng, M, N, d, p, m, n)
    if m > 2:
        bumps[1] = bumps[0]         # duplicated bump
        bumps[2] = tsv[0]           # bump on a TSV
    st = reduced.UniformStack(M, N, r, s, [tuple(t) for t in tsv], Rt)
    ref = reduced.TransformedSystem(st).pairs([tuple(b) for b in bumps], [tuple(l) for l in loads])
    R = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
    stats = er.stack_pairs(M, N, r, s, tsv, Rt, bumps, loads, R)
    got = R.cpu().numpy()
    assert stats["n_system"] == (p + 1) * (d - 1)
    assert stats["wu_pairs"] == d * p * (p - 1) // 2 + (m + n) * p
    rel = np.abs(got - ref) / np.abs(ref)
    assert np.all(np.isfinite(got))
    assert rel.max() <= 1e-9, rel.max()


def test_stack_pairs_invalid(er):
    rng = np.random.default_rng(3)
    r, s, tsv, Rt, bumps, loads = make_stack(rng, 8, 8, 3, 4, 2, 2)
    R = torch.zeros((2, 2), dtype=torch.float64, device="cuda")
    bad = bumps.copy()
    bad[0, 0] = 8
    with pytest.raises(er.ErError):
        er.stack_pairs(8, 8, r, s, tsv, Rt, bad, loads, R)
    with pytest.raises(er.ErError):
        er.stack_pairs(8, 8, r, s, tsv, -Rt, bumps, loads, R)
    with pytest.raises(er.ErError):
        er.stack_pairs(8, 8, r[:1], s[:1], tsv, Rt[:0], bumps, loads, R)  # one die
    er.stack_pairs(8, 8, r, s, tsv, Rt, bumps[:0], loads, R)  # no bumps: no-op
