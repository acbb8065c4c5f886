"""GB300-native preconditioned iPEPS optimisation hot path.

The compute path is the C-ABI library ``libipeps.so`` built from ``csrc/``
(hand-written CUDA for sm_103a).  Importing this package does not load it;
``paper_2511_09546_gb300.ipeps`` does, and raises if it is missing.
"""
