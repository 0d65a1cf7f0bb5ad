"""CPU FP64 oracle for compatible-weighted-matching AMG (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
import this package.  The CUDA path never does.
"""
from .oracle import *  # noqa: F401,F403
