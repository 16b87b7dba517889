"""FP64 CPU oracle for the field-line advection hot path (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It shares no code with the CUDA library.  See
``oracle.c`` for what each function computes and which passage of the paper
it follows.
"""
from .oracle import *  # noqa: F401,F403
