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


def pcg(b, bx, by, bz, periodic=(False, False, False), tol: float = 1e-6, max_iter: int = 10000,
        x0=None, f32_inputs: bool = True, keep_directions: bool = False) -> PcgResult:
    """Jacobi-PCG solve of A x = b (with the projection and the gauge above)."""
    cast = (lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)) if f32_inputs else \
        (lambda a: np.asarray(a, dtype=np.float64))
    b, bx, by, bz = cast(b), cast(bx), cast(by), cast(bz)
    D = jacobi_diagonal(bx, by, bz, periodic)
    active = D > 0.0
    Minv = np.where(active, 1.0 / np.where(active, D, 1.0), 0.0)
    bp = np.where(active, b - (b[active].mean() if active.any() else 0.0), 0.0)
    x = np.zeros_like(bp) if x0 is None else cast(x0).copy()

    def B(v):
        return -O.apply_A(v, bx, by, bz, periodic)

    c = -bp
    bnorm = float(np.linalg.norm(bp))
    res = PcgResult(x, 0, 0, 0.0)
    if bnorm == 0.0:
        res.x = np.zeros_like(bp)
        return res
    r = c - B(x)
    z = Minv * r
    d = z.copy()
    rz = float(np.vdot(r, z))
    rel = float(np.linalg.norm(r)) / bnorm
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
        rel = float(np.linalg.norm(r)) / bnorm
        res.history.append(rel)
    if res.status == 0 and rel > tol:
        res.status = 3
    x = np.where(active, x - (x[active].mean() if active.any() else 0.0), 0.0)
    res.x, res.iterations, res.rel_res = x, k, rel
    return res


def pcg_problem(prob, tol: float = 1e-6, **kw) -> PcgResult:
    return pcg(prob.b, prob.bx, prob.by, prob.bz, prob.periodic, tol=tol, **kw)
