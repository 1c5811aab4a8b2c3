"""GB300-native all-node effective-resistance maps for 3D-IC power delivery networks.

The compute path is the C-ABI library built from ``csrc/`` (hand-written CUDA for
sm_103a); ``er`` is its thin ctypes binding.  ``instances`` draws seeded synthetic
networks.  Importing the package loads nothing; ``paper_2607_05818_gb300.er``
loads the shared library and fails loudly if it is missing.
"""
__all__ = ["instances", "er"]
