"""GB300-native geometric-multigrid pressure-Poisson solver.

The solver runs in hand-written CUDA kernels for sm_103a behind a C ABI
(``include/gmg.h``); this package holds that library's sources (``csrc/``),
its build step (``build.py``), a thin ctypes binding (``binding.py``) and the
seeded synthetic input generators (``inputs.py``).  Importing the package does
not load the library: the binding loads it on first use and raises if it is
missing, so there is no CPU fallback.
"""

__all__ = ["inputs"]
