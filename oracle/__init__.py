"""FP64 CPU oracle for the profile log-likelihood (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package.  The product library never loads it.
"""
from .oracle import *  # noqa: F401,F403
