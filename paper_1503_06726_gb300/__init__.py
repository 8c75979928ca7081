"""GB300 (sm_103a) coupled lattice-Boltzmann / immersed-boundary step of
LBIBCell (arXiv:1503.06726), behind the C ABI of include/lbib.h.

``paper_1503_06726_gb300.lbib`` is the ctypes binding; ``build`` compiles the
CUDA library in-tree.  There is no CPU implementation in this package.
"""
from . import lbib  # noqa: F401
from .lbib import Simulation  # noqa: F401
