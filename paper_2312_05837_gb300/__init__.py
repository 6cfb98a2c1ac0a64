"""GB300 (sm_103a) pruning + domain-selection Ising solver.

The compute path lives in the CUDA library libising_gb300.so (csrc/, C ABI in
include/ising_ds.h); ``api`` is its Python binding. Importing the package loads
the library and raises if it has not been built: there is no CPU fallback.
"""

from . import _lib

_lib.load()

from . import api  # noqa: E402,F401
from .api import Context, IsingError, energy, prune, select_domain, solve, Session  # noqa: E402,F401
