"""The multigrid's coarse levels are networks: the Galerkin product P^T G P equals the
conductance matrix of the 2 x 2-aggregated network (CPU).

For aggregation with piecewise-constant prolongation P (P[i, J] = 1 when fine node i lies in
aggregate J and is not floating), P^T G P is again a network Laplacian plus pads:
- a segment between two aggregates adds its conductance to theirs (parallel ones sum);
- a segment inside an aggregate cancels;
- a TSV segment joins the aggregates of its two ends, which lie on adjacent tiers at the
  same (X, Y);
- a pad moves to its aggregate.
That is the coarsening rule the library applies on the host to build each level.  This
test writes the rule out on the instance arrays and checks it against P^T G P, formed from
the oracle's G.  Shapes are odd, so edge aggregates hold one or two nodes, and the networks
have floating islands.
"""
import os
import sys

import numpy as np
import pytest

from oracle import network
from paper_2607_05818_gb300 import instances as I

sys.path.insert(0, os.path.dirname(__file__))
from mg_rules import aggregate, galerkin  # noqa: E402


CASES = [
    ("ragged_3x7x5", lambda: I.random_small(np.random.default_rng(31), T=3, W=7, H=5, n_tsv=9, n_pads=2)),
    ("floating_1x9x8", lambda: I.random_small(np.random.default_rng(32), T=1, W=9, H=8, n_pads=1, open_frac=0.35)),
    ("even_2x8x6", lambda: I.random_small(np.random.default_rng(33), T=2, W=8, H=6, n_tsv=12, n_pads=3)),
    ("chain_1x11x1", lambda: I.random_small(np.random.default_rng(34), T=1, W=11, H=1, n_pads=1)),
    ("column_4x1x9", lambda: I.random_small(np.random.default_rng(35), T=4, W=1, H=9, n_tsv=8, n_pads=1)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_galerkin_product_is_the_aggregated_network(name, make):
    inst = make()
    coarse = aggregate(inst)
    A = galerkin(inst)
    C = network.conductance_matrix(coarse).toarray()
    assert A.shape == C.shape
    np.testing.assert_allclose(A, C, rtol=1e-12, atol=1e-12 * np.abs(A).max())
    # an aggregate of floating nodes only is floating (an empty row) in the coarse network too
    fl_c = network.floating_mask(coarse)
    empty = np.all(A == 0, axis=1)
    assert np.all(empty <= fl_c)
