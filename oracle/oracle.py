"""Python access to the FP64 CPU oracle, plus closed-form and dense checkers.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module; the solver package never does.

* ``liboracle.so`` (built from ``gmg_oracle.c`` by :func:`build`) is the plain
  FP64 V-cycle / adaptive-omega RBGS / iso-aniso coarsening solver of the
  paper's Sec. 3, 3.1 and 3.2 (readings C1-C8 in the C file's header).
* :func:`fft_solve_periodic` is the exact discrete solution of the uniform
  triple-periodic problem (C9): p_hat(k) = b_hat(k) / lambda(k) with
  lambda(k) = -sum_d 4 sin^2(pi k_d / n_d), p_hat(0) = 0.
* :func:`dense_operator` assembles the 7-point face-flux matrix from the
  definition of the problem (sum over faces of beta_f (p_nb - p_I)) with
  scipy, independently of the C oracle, for the brute-force pins on tiny grids.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gmg_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

OK, ERR_ARG, NOT_CONVERGED, DIVERGED = 0, 1, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE arithmetic, no contraction)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared",
                               "-fPIC", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Options(ctypes.Structure):
    _fields_ = [("coarsen", ctypes.c_int), ("n_min", ctypes.c_int), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("nu_c", ctypes.c_int), ("max_cycles", ctypes.c_int),
                ("omega0", ctypes.c_double), ("omega_min", ctypes.c_double),
                ("shrink", ctypes.c_double), ("grow", ctypes.c_double), ("coarse_mode", ctypes.c_int),
                ("coarse_op", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("status", ctypes.c_int), ("levels", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("omega", ctypes.c_double),
                ("bnorm", ctypes.c_double)]


def options(coarsen: str = "aniso", n_min: int = 4, nu1: int = 2, nu2: int = 2, nu_c: int = 16,
            max_cycles: int = 100, omega0: float = 1.0, omega_min: float = 0.25,
            shrink: float = 0.7, grow: float = 1.1, coarse_mode: int = 0, coarse_op: int = 0) -> Options:
    """coarse_mode 0: nu_c sweeps on the coarsest level; 1: its minimum-norm dense solve.
    coarse_op 0: finite-volume coarse coefficients; 1: Galerkin R A P (C4's option)."""
    return Options(1 if coarsen == "aniso" else 0, n_min, nu1, nu2, nu_c, max_cycles,
                   omega0, omega_min, shrink, grow, coarse_mode, coarse_op)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        I = ctypes.POINTER(ctypes.c_int)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        _lib.or_solve.argtypes = [c_int, c_int, c_int, I, ctypes.POINTER(Options), D, D, D, D, D,
                                  c_double, ctypes.POINTER(_Info), D, D, I]
        _lib.or_apply_A.argtypes = [c_int, c_int, c_int, I, D, D, D, D, D]
        _lib.or_half_sweep.argtypes = [c_int, c_int, c_int, I, D, D, D, D, D, c_double, c_int]
        _lib.or_sweep.argtypes = [c_int, c_int, c_int, I, D, D, D, D, D, c_double]
        _lib.or_schedule.argtypes = [c_int, c_int, c_int, I, c_int, c_int, I, I]
        _lib.or_coarsen_beta.argtypes = [c_int, c_int, c_int, I, I, D, D, D, D, D, D, c_int]
        _lib.or_restrict.argtypes = [c_int, c_int, c_int, I, D, D]
        _lib.or_prolong_add.argtypes = [c_int, c_int, c_int, I, D, D]
        _lib.or_vcycle.argtypes = [c_int, c_int, c_int, I, ctypes.POINTER(Options), D, D, D, D, D,
                                   c_double]
        _lib.or_pinv_apply.argtypes = [c_int, c_int, c_int, I, D, D, D, D, D]
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ivec(v):
    arr = (ctypes.c_int * len(v))(*[int(x) for x in v])
    return arr


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _dims(a: np.ndarray):
    nz, ny, nx = a.shape
    return nx, ny, nz


def apply_A(p, bx, by, bz, periodic=(False, False, False)) -> np.ndarray:
    p, bx, by, bz = map(_f64, (p, bx, by, bz))
    out = np.empty_like(p)
    lib().or_apply_A(*_dims(p), _ivec(periodic), _d(bx), _d(by), _d(bz), _d(p), _d(out))
    return out


def half_sweep(p, b, bx, by, bz, omega, colour, periodic=(False, False, False)) -> np.ndarray:
    p = _f64(p).copy()
    b, bx, by, bz = map(_f64, (b, bx, by, bz))
    lib().or_half_sweep(*_dims(p), _ivec(periodic), _d(bx), _d(by), _d(bz), _d(b), _d(p),
                        float(omega), int(colour))
    return p


def sweep(p, b, bx, by, bz, omega, periodic=(False, False, False)) -> np.ndarray:
    p = _f64(p).copy()
    b, bx, by, bz = map(_f64, (b, bx, by, bz))
    lib().or_sweep(*_dims(p), _ivec(periodic), _d(bx), _d(by), _d(bz), _d(b), _d(p), float(omega))
    return p


def schedule(dims, periodic=(False, False, False), coarsen: str = "aniso", n_min: int = 4):
    d = (ctypes.c_int * 96)()
    f = (ctypes.c_int * 96)()
    L = lib().or_schedule(int(dims[0]), int(dims[1]), int(dims[2]), _ivec(periodic),
                          1 if coarsen == "aniso" else 0, n_min, d, f)
    return ([tuple(d[3 * l:3 * l + 3]) for l in range(L)],
            [tuple(f[3 * l:3 * l + 3]) for l in range(L)])


def coarsen_beta(bx, by, bz, fac, periodic=(False, False, False), galerkin: bool = False):
    bx, by, bz = map(_f64, (bx, by, bz))
    nz, ny, nx = bx.shape
    cshape = (nz // fac[2], ny // fac[1], nx // fac[0])
    out = [np.empty(cshape) for _ in range(3)]
    lib().or_coarsen_beta(nx, ny, nz, _ivec(periodic), _ivec(fac), _d(bx), _d(by), _d(bz),
                          *[_d(o) for o in out], int(bool(galerkin)))
    return tuple(out)


def restrict(r, fac) -> np.ndarray:
    r = _f64(r)
    nz, ny, nx = r.shape
    out = np.empty((nz // fac[2], ny // fac[1], nx // fac[0]))
    lib().or_restrict(nx, ny, nz, _ivec(fac), _d(r), _d(out))
    return out


def prolong_add(p, e, fac) -> np.ndarray:
    p = _f64(p).copy()
    e = _f64(e)
    nz, ny, nx = p.shape
    lib().or_prolong_add(nx, ny, nz, _ivec(fac), _d(e), _d(p))
    return p


def vcycle(p, b, bx, by, bz, omega=1.0, periodic=(False, False, False), **opt) -> np.ndarray:
    p = _f64(p).copy()
    b, bx, by, bz = map(_f64, (b, bx, by, bz))
    o = options(**opt)
    lib().or_vcycle(*_dims(p), _ivec(periodic), ctypes.byref(o), _d(bx), _d(by), _d(bz), _d(b),
                    _d(p), float(omega))
    return p


def pinv_apply(b, bx, by, bz, periodic=(False, False, False)) -> np.ndarray:
    """The dense coarsest-level step (coarse_mode 1) on one grid: p = A^+ b."""
    b, bx, by, bz = map(_f64, (b, bx, by, bz))
    p = np.empty_like(b)
    lib().or_pinv_apply(*_dims(b), _ivec(periodic), _d(bx), _d(by), _d(bz), _d(b), _d(p))
    return p


@dataclass
class Result:
    p: np.ndarray
    cycles: int
    status: int
    levels: int
    rel_res: float
    omega: float
    bnorm: float
    history: np.ndarray        # relative residual of the accepted iterate, per cycle
    omegas: np.ndarray         # omega used by each cycle
    accepted: np.ndarray       # accept flag of each cycle


def solve(b, bx, by, bz, periodic=(False, False, False), tol: float = 1e-6, p0=None,
          **opt) -> Result:
    """Full oracle solve (C5-C8).  Inputs are cast to float64."""
    b, bx, by, bz = map(_f64, (b, bx, by, bz))
    p = np.zeros_like(b) if p0 is None else _f64(p0).copy()
    o = options(**opt)
    n = o.max_cycles
    hr = np.zeros(n + 1)
    ho = np.zeros(max(n, 1))
    ha = np.zeros(max(n, 1), dtype=np.int32)
    info = _Info()
    rc = lib().or_solve(*_dims(b), _ivec(periodic), ctypes.byref(o), _d(bx), _d(by), _d(bz), _d(b),
                        _d(p), float(tol), ctypes.byref(info), _d(hr), _d(ho),
                        ha.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if rc != OK:
        raise ValueError(f"oracle solve rejected its arguments (code {rc})")
    k = info.cycles
    return Result(p, k, info.status, info.levels, info.rel_res, info.omega, info.bnorm,
                  hr[:k + 1].copy(), ho[:k].copy(), ha[:k].astype(bool))


def solve_problem(prob, tol: float = 1e-6, f32_inputs: bool = True, **opt) -> Result:
    """Oracle solve of an ``inputs.Problem``; by default on its float32-rounded inputs."""
    cast = (lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)) if f32_inputs else _f64
    return solve(cast(prob.b), cast(prob.bx), cast(prob.by), cast(prob.bz), prob.periodic,
                 tol=tol, **opt)


# ----------------------------------------------------------------------------
# Closed forms and brute force, independent of the C oracle
# ----------------------------------------------------------------------------

def fft_solve_periodic(b) -> np.ndarray:
    """Exact discrete solution for beta = 1 on a triple-periodic grid (C9)."""
    b = _f64(b)
    nz, ny, nx = b.shape
    lam = np.zeros((nz, ny, nx // 2 + 1))
    for axis, n in ((0, nz), (1, ny), (2, nx)):
        k = np.arange(n if axis < 2 else nx // 2 + 1)
        l1 = -4.0 * np.sin(np.pi * k / n) ** 2
        shape = [1, 1, 1]
        shape[axis] = len(k)
        lam = lam + l1.reshape(shape)
    bh = np.fft.rfftn(b - b.mean())
    lam[0, 0, 0] = 1.0
    ph = bh / lam
    ph[0, 0, 0] = 0.0
    return np.fft.irfftn(ph, s=b.shape, axes=(0, 1, 2))


def dense_operator(bx, by, bz, periodic=(False, False, False)):
    """Assemble the face-flux operator as a dense matrix by looping over faces.

    Every face with coefficient beta between cells P and Q adds the 2x2 block
    beta * [[-1, 1], [1, -1]]; this is the conservative finite-volume
    definition, written face by face rather than cell by cell.
    """
    bx, by, bz = map(_f64, (bx, by, bz))
    nz, ny, nx = bx.shape
    N = nx * ny * nz
    A = np.zeros((N, N))

    def cell(i, j, k):
        return (k * ny + j) * nx + i

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for axis, beta, n, lo in ((0, bx, nx, i), (1, by, ny, j), (2, bz, nz, k)):
                    # lower face of (i, j, k) on this axis
                    if lo == 0 and not periodic[axis]:
                        continue
                    q = [i, j, k]
                    q[axis] = (lo - 1) % n
                    P, Q = cell(i, j, k), cell(*q)
                    f = beta[k, j, i]
                    A[P, P] -= f
                    A[Q, Q] -= f
                    A[P, Q] += f
                    A[Q, P] += f
    return A


def dense_solve(b, bx, by, bz, periodic=(False, False, False)) -> np.ndarray:
    """Minimum-norm least-squares solution of A p = b (projected) on a tiny grid."""
    import scipy.linalg
    A = dense_operator(bx, by, bz, periodic)
    p, *_ = scipy.linalg.lstsq(A, _f64(b).ravel(), lapack_driver="gelsd")
    return p.reshape(np.shape(b))
