"""CPU oracle for sparse-oblique split search (test infrastructure only).

Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never imports it.
"""
from .so_oracle import *  # noqa: F401,F403
