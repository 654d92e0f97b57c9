"""FP64 CPU oracle for GAP-TV / ADMM-TV video SCI reconstruction.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
never calls it, and it never calls the CUDA library: the two share no code.
"""
from .sci_oracle import *  # noqa: F401,F403
from .sci_oracle import __all__  # noqa: F401
from . import lprox_oracle  # noqa: F401
