"""CPU oracle for the matrix-free Heisenberg product (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
Python binding) never does.
"""
from .oracle import *  # noqa: F401,F403
