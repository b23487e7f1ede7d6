"""CPU FP64 oracle -- TEST INFRASTRUCTURE, not part of the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  It shares
no code with the CUDA library under ``paper_1407_3535_gb300/`` and neither
imports the other.

``oracle.ref`` holds the definitions (numpy + a small C library compiled
from ``oracle/zncc_ref.c``).  Every function is pinned by the ``-m "not gpu"``
tests in ``tests/test_oracle_pins.py`` against something other than itself:
exact rational arithmetic, closed forms and invariants of Eq. rho1, the
values the paper prints (Fig. 2, Eq. misDec), library routines (a Gaussian
filter, corrcoef), brute force on tiny inputs, and constructed images whose
answer is known by design (the block the level loop of Algorithm 3 must
freeze).  The FFT form of the full map is pinned to the direct definition.
"""
