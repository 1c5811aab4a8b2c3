"""CPU oracle for all-node effective-resistance maps (test infrastructure only).

This package is the slow, obviously correct FP64 reference that the CUDA path is
checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the
product library never does, and it never imports the product library.  Its
inputs are plain arrays (the attributes of a network instance: T, W, H, gx, gy,
tsv_*, pad_*), drawn by the seeded generator that both sides share.

Modules and what they follow:
  network  canonical edge list, G = B^T W B + D (Eq. 1 form), floating nodes
  exact    diag(G^-1) by dense Cholesky, Gauss-Jordan brute force, the Eq. 2
           pseudo-inverse route, sampled direct solves for large networks
  sketch   the counter-based Rademacher JL sketch Y^T = M^T Q^T and R_JL
  wu       Wu's two-point resistance of a uniform free-boundary mesh (Eq. 3)
  reduced  the paper's reduced TSV system (Eq. 6-12) and its transformed,
           pair-independent form (Eq. 13-15)
  pairs    pairwise R (Eq. 2 / Eq. 4 on the grounded network) and IR drop
           G^-1 I (Eq. 1), exact and as same-seed JL estimates from Z

Every function here is pinned by a test in tests/test_oracle_pins.py against a
closed form, an identity or brute force; none is "parity unpinned".
"""
