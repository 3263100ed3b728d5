"""Exact multi-modular resultants and gcds on GB300 (sm_103a).

The compute path is libgbres.so (CUDA kernels behind the C ABI in
include/gbres.h); this package holds its build script, the thin Python binding
(``api``) and the seeded input generators (``workloads``).  Importing the
package does not load the library; creating a :class:`Context` does, and fails
loudly if the library or the GPU is missing.
"""

from .build import build  # noqa: F401


def __getattr__(name):
    if name in ("Context", "Resident", "resultant_info", "primes"):
        from . import api

        return getattr(api, name)
    raise AttributeError(name)
