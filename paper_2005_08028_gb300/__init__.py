"""GAP-TV / ADMM-TV video snapshot compressive imaging reconstruction on GB300.

The compute lives in libsci.so (CUDA, sm_103a; C ABI in include/sci.h).
``paper_2005_08028_gb300.sci`` is the Python binding; ``build`` compiles the
library in-tree.
"""
from . import sci  # noqa: F401
from .sci import *  # noqa: F401,F403
