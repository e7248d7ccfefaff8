"""GB300-native geometric-multigrid pressure-Poisson solver.

The solver runs in hand-written CUDA kernels for sm_103a behind a C ABI
(``include/gmg.h``, ``include/gmg_net.h``); this package holds that library's
sources (``csrc/``), its build step (``build.py``), a thin ctypes binding
(``binding.py``), the learned warm start built on the network kernels
(``warmstart.py``) and the seeded synthetic input generators (``inputs.py``).
Importing the package does not load the library: the binding loads it on first
use and raises if it is missing, so there is no CPU fallback.

Typical use (device tensors of nx*ny*nz, x fastest)::

    from paper_2607_07687_gb300 import binding as G
    with G.Solver((nx, ny, nz), periodic=(False, False, False),
                  coarsen="aniso", precision="ir64_fp32") as s:
        s.set_coeffs(bx, by, bz)          # float32 lower-face coefficients
        info = s.solve(sigma64, p64, 1e-6)  # FP64 refinement around FP32 V-cycles
    # G.BatchSolver: many problems per launch; s.pcg_solve / s.gmgpcg_solve:
    # the paper's comparison solvers on an FP32 handle; G.tune_export /
    # G.tune_import: the autotuner's launch shapes across processes.
"""

__all__ = ["inputs"]
