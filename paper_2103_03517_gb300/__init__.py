"""GB300 (sm_103a) implementation of the parallel checkerboard and parallel
constrained Metropolis Monte Carlo algorithms of Lepadatu et al.
(arXiv:2103.03517) for the classical Heisenberg model on a simple-cubic
lattice.

The compute path is the CUDA library libmc.so (C ABI in include/mc.h);
``paper_2103_03517_gb300._mc`` binds its entry points under the same names.
"""
from ._mc import *  # noqa: F401,F403
from ._mc import lib  # noqa: F401
