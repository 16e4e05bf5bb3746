"""FP64 CPU oracle of the OpenCFD-SCU stage right-hand side and TVD-RK3 step.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The oracle shares no
code with the CUDA path (arXiv:2209.15333, Sections 2.1-2.4).

Parity pins: every part of the oracle is checked in ``tests/test_oracle_*.py``
against closed forms, textbook special cases, the paper's printed coefficients
(Eq. 41) and brute-force symbolic computations.
"""
from .oracle import *  # noqa: F401,F403
