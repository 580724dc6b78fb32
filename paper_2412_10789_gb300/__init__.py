"""GB300-native ChebyPower: graph propagation (SSPPR / HKPR) by the Chebyshev
power iteration of arXiv 2412.10789, as a C-ABI CUDA library for sm_103a.

``paper_2412_10789_gb300.gp`` is the ctypes binding of ``include/gp.h``;
``paper_2412_10789_gb300.build`` compiles ``csrc/`` into ``libgpcheby.so``.
"""
from .gp import *  # noqa: F401,F403
from .gp import load_library  # noqa: F401
