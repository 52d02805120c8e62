"""VOiLA rollout and belief-update hot path for B300 (sm_103a).

The compute path lives in the C-ABI shared library built from ``csrc/``;
``voila`` is its thin ctypes binding. Importing this package does not load
the library; ``paper_2606_19729_b300.voila`` does, and raises if it is
missing.
"""
