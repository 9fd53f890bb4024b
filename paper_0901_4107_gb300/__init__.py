"""GB300-native moving-mesh hydrodynamics: one MUSCL-Hancock update of the
ideal-gas Euler equations on a given Voronoi tessellation (Springel 2010,
Sec. 3), as hand-written CUDA for sm_103a behind the C ABI of include/amm.h.

`paper_0901_4107_gb300.amm` is the ctypes binding (same names as the C
calls).  The library is built in-tree by `__graft_entry__.build()`.
"""
from . import amm  # noqa: F401
