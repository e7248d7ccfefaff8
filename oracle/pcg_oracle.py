"""pcg_oracle.py -- plain FP64 reference of the Jacobi-preconditioned conjugate-
gradient Poisson solve: the general-purpose solver the paper compares its
multigrid against (Sec. 3: PCG applies to any grid but needs global inner
products every iteration; Table 1).

TEST INFRASTRUCTURE ONLY.  This is the checker of the GPU conjugate-gradient
solver; it shares no code with it, and only the tests, the smoke check and the
benchmark's CPU leg may use it.  The operator is the multigrid oracle's own
FP64 apply (oracle.apply_A), pinned by its tests.

Readings (the paper names PCG, nothing more):
  C14 preconditioner  Jacobi: M = diag(-A), the sum of a cell's open face
                      coefficients; cells with no open face are left out
                      (M^-1 = 0 there, so they never change).
  projection, gauge   as for the multigrid solve: b <- b - mean over active
                      cells and 0 on inactive cells; at exit the iterate's mean
                      over active cells is removed and inactive cells are 0.
  stop                |r_k| / |b| <= tol with r_k the recursively updated
                      residual, or max_iter iterations.

Algorithm: preconditioned conjugate gradients (Hestenes and Stiefel with a
preconditioner, as in Saad, Iterative Methods for Sparse Linear Systems,
Alg. 9.1) on the symmetric positive semi-definite system B x = c with B = -A,
c = -b, from x0:
  r0 = c - B x0,  z0 = M^-1 r0,  d0 = z0
  alpha_k = (r_k, z_k) / (d_k, B d_k)
  x_{k+1} = x_k + alpha_k d_k,   r_{k+1} = r_k - alpha_k B d_k
  z_{k+1} = M^-1 r_{k+1},        beta_k = (r_{k+1}, z_{k+1}) / (r_k, z_k)
  d_{k+1} = z_{k+1} + beta_k d_k
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import oracle as O


@dataclass
class PcgResult:
    x: np.ndarray
    iterations: int
    status: int                    # 0 converged, 3 max_iter reached, 4 breakdown
    rel_res: float                 # |r| / |b| of the last iterate (recursive residual)
    history: List[float] = field(default_factory=list)
    directions: List[np.ndarray] = field(default_factory=list)


def faces(bx, by, bz, periodic=(False, False, False)):
    """Lower and upper face coefficients of every cell, walls closed.  Arrays are
    (nz, ny, nx); the lower x face of cell I is bx[I]."""
    lo = []
    up = []
    for d, (b, axis) in enumerate(((bx, 2), (by, 1), (bz, 0))):
        b = np.array(b, dtype=np.float64)
        if not periodic[d]:
            idx = [slice(None)] * 3
            idx[axis] = 0
            b[tuple(idx)] = 0.0          # the lower boundary face is a wall
        u = np.roll(b, -1, axis=axis)    # upper face of I = lower face of I + e_d
        if not periodic[d]:
            idx = [slice(None)] * 3
            idx[axis] = -1
            u[tuple(idx)] = 0.0          # the upper boundary face is a wall
        lo.append(b)
        up.append(u)
    return lo, up


def jacobi_diagonal(bx, by, bz, periodic=(False, False, False)) -> np.ndarray:
    """diag(-A): the sum of the six face coefficients of each cell (C14)."""
    lo, up = faces(bx, by, bz, periodic)
    return (lo[0] + up[0]) + (lo[1] + up[1]) + (lo[2] + up[2])


def _cg(x, b, bx, by, bz, periodic, tol, max_iter, bnorm=None, keep_directions=False) -> PcgResult:
    """The iteration itself: PCG on B x = -b (B = -A) from x, stopping when
    |r| / bnorm <= tol or after max_iter steps; bnorm None: relative to |r_0|."""
    D = jacobi_diagonal(bx, by, bz, periodic)
    active = D > 0.0
    Minv = np.where(active, 1.0 / np.where(active, D, 1.0), 0.0)

    def B(v):
        return -O.apply_A(v, bx, by, bz, periodic)

    res = PcgResult(x, 0, 0, 0.0)
    r = -b - B(x)
    z = Minv * r
    d = z.copy()
    rz = float(np.vdot(r, z))
    if bnorm is None:
        bnorm = float(np.linalg.norm(r))
    rel = float(np.linalg.norm(r)) / bnorm if bnorm > 0 else 0.0
    res.history.append(rel)
    k = 0
    while rel > tol and k < max_iter:
        if keep_directions:
            res.directions.append(d.copy())
        w = B(d)
        dw = float(np.vdot(d, w))
        if not dw > 0.0:
            res.status = 4
            break
        alpha = rz / dw
        x = x + alpha * d
        r = r - alpha * w
        z = Minv * r
        rz_new = float(np.vdot(r, z))
        beta = rz_new / rz
        rz = rz_new
        d = z + beta * d
        k += 1
        rel = float(np.linalg.norm(r)) / bnorm if bnorm > 0 else 0.0
        res.history.append(rel)
    if res.status == 0 and rel > tol:
        res.status = 3
    res.x, res.iterations, res.rel_res = x, k, rel
    return res


def _project(b, active):
    return np.where(active, b - (b[active].mean() if active.any() else 0.0), 0.0)


def pcg(b, bx, by, bz, periodic=(False, False, False), tol: float = 1e-6, max_iter: int = 10000,
        x0=None, f32_inputs: bool = True, keep_directions: bool = False) -> PcgResult:
    """Jacobi-PCG solve of A x = b (with the projection and the gauge above)."""
    cast = (lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)) if f32_inputs else \
        (lambda a: np.asarray(a, dtype=np.float64))
    b, bx, by, bz = cast(b), cast(bx), cast(by), cast(bz)
    active = jacobi_diagonal(bx, by, bz, periodic) > 0.0
    bp = _project(b, active)
    x = np.zeros_like(bp) if x0 is None else cast(x0).copy()
    bnorm = float(np.linalg.norm(bp))
    if bnorm == 0.0:
        return PcgResult(np.zeros_like(bp), 0, 0, 0.0)
    res = _cg(x, bp, bx, by, bz, periodic, tol, max_iter, bnorm, keep_directions)
    res.x = _project(res.x, active)      # the gauge: mean over active cells removed
    return res


# ---------------------------------------------------------------- GMG-PCG
#
# The multigrid of the paper with PCG as its smoother ("GMG-PCG", Table 1).
# Readings: the V-cycle, hierarchy, transfers and coarse coefficients are the
# RBGS cycle's (C3, C4, C6); each smoothing step is a fresh Jacobi-PCG run of
# nu1 (before), nu2 (after) or nu_c (coarsest) iterations on the level's
# equation from the level's current iterate, with no gauge inside the cycle
# and the coarsest right-hand side projected to zero mean as in C6; a
# smoothing run also ends once its residual has fallen to
# SMOOTH_ETA of its start (CG has then solved the level: further steps would
# divide rounding noise by rounding noise); a V-cycle is always accepted
# (there is no relaxation factor to adapt); the solve stops when
# |b - A x| / |b| <= tol.
SMOOTH_ETA = 1e-10


def gmg_pcg_vcycle(x, b, levels, l, nu1, nu2, nu_c, periodic):
    """One V-cycle from level l; levels[k] = (bx, by, bz, fac to k + 1)."""
    bx, by, bz, fac = levels[l]
    if l == len(levels) - 1:
        # the coarsest right-hand side projected to zero mean over active cells (C6):
        # CG on the singular coarsest operator needs a consistent right-hand side
        active = jacobi_diagonal(bx, by, bz, periodic) > 0.0
        return _cg(x, _project(b, active), bx, by, bz, periodic, SMOOTH_ETA, nu_c).x
    x = _cg(x, b, bx, by, bz, periodic, SMOOTH_ETA, nu1).x
    r = b - O.apply_A(x, bx, by, bz, periodic)
    bc = O.restrict(r, fac)
    ec = gmg_pcg_vcycle(np.zeros_like(bc), bc, levels, l + 1, nu1, nu2, nu_c, periodic)
    x = O.prolong_add(x, ec, fac)
    return _cg(x, b, bx, by, bz, periodic, SMOOTH_ETA, nu2).x


def hierarchy(bx, by, bz, periodic, coarsen, n_min):
    dims = (bx.shape[2], bx.shape[1], bx.shape[0])
    _, facs = O.schedule(dims, periodic, coarsen=coarsen, n_min=n_min)
    levels, beta = [], (bx, by, bz)
    for l, f in enumerate(facs):
        levels.append((beta[0], beta[1], beta[2], f))
        if l + 1 < len(facs):
            beta = O.coarsen_beta(*beta, f, periodic)
    return levels


def gmg_pcg_solve(b, bx, by, bz, periodic=(False, False, False), tol: float = 1e-6, coarsen: str = "aniso",
                  n_min: int = 4, nu1: int = 2, nu2: int = 2, nu_c: int = 16, max_cycles: int = 100,
                  f32_inputs: bool = True) -> PcgResult:
    """GMG-PCG solve from a zero guess (projection and gauge as for the other solvers);
    iterations = V-cycles, history = relative residual before each cycle and at the end."""
    cast = (lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)) if f32_inputs else \
        (lambda a: np.asarray(a, dtype=np.float64))
    b, bx, by, bz = cast(b), cast(bx), cast(by), cast(bz)
    active = jacobi_diagonal(bx, by, bz, periodic) > 0.0
    bp = _project(b, active)
    bnorm = float(np.linalg.norm(bp))
    x = np.zeros_like(bp)
    res = PcgResult(x, 0, 0, 0.0)
    if bnorm == 0.0:
        return res
    levels = hierarchy(bx, by, bz, periodic, coarsen, n_min)
    k = 0
    while True:
        rel = float(np.linalg.norm(bp - O.apply_A(x, bx, by, bz, periodic))) / bnorm
        res.history.append(rel)
        if rel <= tol or k >= max_cycles:
            break
        x = gmg_pcg_vcycle(x, bp, levels, 0, nu1, nu2, nu_c, periodic)
        k += 1
    res.status = 0 if rel <= tol else 3
    res.x, res.iterations, res.rel_res = _project(x, active), k, rel
    return res


def pcg_problem(prob, tol: float = 1e-6, **kw) -> PcgResult:
    return pcg(prob.b, prob.bx, prob.by, prob.bz, prob.periodic, tol=tol, **kw)
