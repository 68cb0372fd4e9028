"""GB300 (sm_103a) particle forward maps for sparse-observation inverse problems.

Implements the particle methods of Borggaard, Glatt-Holtz & Krometis
(arXiv:1808.10580): the parameter-to-observation map G(u) evaluated by
independent backward Euler-Maruyama particles, for the time-dependent
advection-diffusion problem (Algorithm 1) and the Dirichlet problem
(Algorithm 2).  The compute runs in hand-written CUDA kernels behind the C ABI
of ``include/pm.h``; ``_lib`` is its thin ctypes binding and ``inputs`` holds
the seeded synthetic workloads.  Loading the CUDA library is deferred to the
first call, and fails loudly if it is missing.
"""
from . import inputs  # noqa: F401
from ._lib import *  # noqa: F401,F403
from ._lib import load  # noqa: F401
