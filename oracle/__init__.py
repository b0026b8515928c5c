"""FP64 CPU oracle (test infrastructure only).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of bench.py
may import this package.  The library never does, and the oracle never
imports the library: the only code both sides share is the seeded input
generator module, which contains no solver arithmetic.
"""
from .kop_oracle import *  # noqa: F401,F403
from . import kop_oracle  # noqa: F401
