"""CPU FP64 oracle -- TEST INFRASTRUCTURE, not part of the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg (and its ``--impl reference`` arm) may import this package.  It shares
no code with the CUDA library under ``paper_1407_3535_gb300/`` and neither
imports the other.

``oracle.ref`` holds the definitions (numpy + a small C library compiled
from ``oracle/zncc_ref.c``).  Parity of every function is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_pins.py``; the one function
without an independent pin is marked "parity unpinned" in its docstring.
"""
