"""Plain FP64 CPU oracle of the saliency method (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import
this package.  The product path (the CUDA library and its binding) never does.
"""
from .oracle import *  # noqa: F401,F403
