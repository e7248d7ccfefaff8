"""ctypes binding of ``libgmg.so`` (the C ABI declared in ``include/gmg.h``).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  Grid arrays are torch tensors on the CUDA device (C-contiguous,
shape ``(nz, ny, nx)``), passed by data pointer on the current torch stream
unless a stream is given.  The library is loaded on first use; if it is
missing or cannot be loaded this module raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import re
from dataclasses import dataclass
from typing import List, Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgmg.so")
HEADER = os.path.join(HERE, "..", "include", "gmg.h")
NET_HEADER = os.path.join(HERE, "..", "include", "gmg_net.h")

OK, ERR_ARG, ERR_CUDA, NOT_CONVERGED, DIVERGED, NONFINITE = 0, 1, 2, 3, 4, 5
STATUS_NAMES = {OK: "ok", ERR_ARG: "bad argument", ERR_CUDA: "cuda error",
                NOT_CONVERGED: "not converged", DIVERGED: "diverged", NONFINITE: "non-finite source"}
ISO, ANISO = 0, 1
COARSE_SWEEPS, COARSE_DENSE = 0, 1
COARSE_OP_FV, COARSE_OP_GALERKIN = 0, 1
FP32, FP32_BF16, IR64, IR64_FP32 = 0, 1, 2, 3
PRECISIONS = {"fp32": FP32, "fp32_bf16": FP32_BF16, "ir64": IR64, "ir64_fp32": IR64_FP32}


class Options(ctypes.Structure):
    _fields_ = [("coarsen", ctypes.c_int), ("n_min", ctypes.c_int), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("nu_c", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_cycles", ctypes.c_int), ("omega0", ctypes.c_double),
                ("omega_min", ctypes.c_double), ("shrink", ctypes.c_double),
                ("grow", ctypes.c_double), ("use_graph", ctypes.c_int),
                ("cycles_per_sync", ctypes.c_int), ("ir_inner_rtol", ctypes.c_double),
                ("autotune", ctypes.c_int), ("coarse_mode", ctypes.c_int), ("coarse_op", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("cycles", ctypes.c_int), ("status", ctypes.c_int), ("levels", ctypes.c_int),
                ("outer", ctypes.c_int), ("launches", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("omega", ctypes.c_double),
                ("bnorm", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class GmgError(RuntimeError):
    pass


_lib = None


def library_path() -> str:
    return LIB_PATH


def lib() -> ctypes.CDLL:
    """Load libgmg.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise GmgError(f"{LIB_PATH} is missing: build it with paper_2607_07687_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    c_int, c_double = ctypes.c_int, ctypes.c_double
    L.gmg_default_options.argtypes = [ctypes.POINTER(Options)]
    L.gmg_default_options.restype = None
    L.gmg_create.argtypes = [ctypes.POINTER(vp), c_int, c_int, c_int, ip, ctypes.POINTER(Options), vp]
    L.gmg_set_coeffs.argtypes = [vp, vp, vp, vp]
    L.gmg_solve.argtypes = [vp, vp, vp, c_double, ctypes.POINTER(Info)]
    L.gmg_solve_host.argtypes = [vp, vp, vp, c_double, ctypes.POINTER(Info)]
    L.gmg_pcg_solve.argtypes = [vp, vp, vp, c_double, c_int, ctypes.POINTER(Info)]
    L.gmg_gmgpcg_solve.argtypes = [vp, vp, vp, c_double, ctypes.POINTER(Info)]
    L.gmg_history.argtypes = [vp, dp, dp, ip, c_int]
    L.gmg_levels.argtypes = [vp, ip]
    L.gmg_bottom_form.argtypes = [vp, ip, ip]
    L.gmg_destroy.argtypes = [vp]
    L.gmg_last_error.argtypes = [vp]
    L.gmg_last_error.restype = ctypes.c_char_p
    L.gmg_batch_create.argtypes = [ctypes.POINTER(vp), c_int, ip, ip, ctypes.POINTER(Options), vp]
    L.gmg_batch_set_coeffs.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.gmg_batch_solve.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), c_double, ctypes.POINTER(Info)]
    L.gmg_batch_destroy.argtypes = [vp]
    L.gmg_batch_last_error.argtypes = [vp]
    L.gmg_batch_last_error.restype = ctypes.c_char_p
    L.gmg_op_sweep.argtypes = [c_int, c_int, c_int, ip, vp, vp, vp, vp, vp, vp, c_double, vp]
    L.gmg_op_sweep_reference.argtypes = [c_int, c_int, c_int, ip, vp, vp, vp, vp, vp, c_double, vp]
    L.gmg_op_residual_restrict.argtypes = [c_int, c_int, c_int, ip, ip, vp, vp, vp, vp, vp, vp, dp, vp]
    L.gmg_op_prolong_add.argtypes = [c_int, c_int, c_int, ip, vp, vp, vp]
    L.gmg_op_residual64.argtypes = [c_int, c_int, c_int, ip, vp, vp, vp, vp, vp, vp, vp, dp, c_int, vp]
    L.gmg_op_coarsen_coeffs.argtypes = [c_int, c_int, c_int, ip, ip, vp, vp, vp, vp, vp, vp, vp]
    L.gmg_op_residual_norm.argtypes = [c_int, c_int, c_int, ip, vp, vp, vp, vp, vp, dp, vp]
    L.gmg_op_residual_norm_noalloc.argtypes = [c_int, c_int, c_int, ip, vp, vp, vp, vp, vp, dp, vp]
    L.gmg_test_poison_omega.argtypes = [vp, c_int]
    L.gmg_test_ring_wait_tries.argtypes = [c_int]
    L.gmg_test_cluster_ranks.argtypes = [c_int]
    L.gmg_tune_export.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.gmg_tune_import.argtypes = [ctypes.c_char_p]
    _net_signatures(L)
    _lib = L
    return L


def _net_signatures(L):
    vp, c_int, c_float, c_ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_longlong
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "gmg_net_conv3": [c_int, c_int, c_int, vp, c_int, c_int, vp, vp, c_int, c_int, vp, c_int, c_int, vp],
        "gmg_net_conv3_wgrad": [c_int, c_int, c_int, vp, c_int, c_int, vp, c_int, c_int, vp, vp, vp],
        "gmg_net_relu_backward": [c_int, c_int, c_int, vp, c_int, vp, c_int, c_int, vp],
        "gmg_net_pool2": [c_int, c_int, c_int, vp, c_int, c_int, vp, c_int, c_int, vp],
        "gmg_net_pool2_backward": [c_int, c_int, c_int, vp, c_int, c_int, vp, c_int, vp, c_int, c_int, vp],
        "gmg_net_up2": [c_int, c_int, c_int, vp, c_int, c_int, vp, c_int, c_int, vp],
        "gmg_net_up2_backward": [c_int, c_int, c_int, vp, c_int, c_int, c_int, vp, c_int, vp],
        "gmg_net_pack_input": [c_int, c_int, c_int, vp, vp, vp, vp, vp, ip, vp, vp, vp, vp],
        "gmg_net_head": [c_int, c_int, c_int, vp, c_int, vp, vp, vp, vp],
        "gmg_net_loss": [c_int, c_int, c_int, vp, vp, vp, vp, vp, vp, vp, vp],
        "gmg_net_residual_loss": [c_int, c_int, c_int, vp, vp, vp, vp, vp, vp, vp, ip, vp, vp, vp, vp, vp],
        "gmg_net_head_backward": [c_int, c_int, c_int, vp, vp, c_int, vp, vp, vp, vp, vp],
        "gmg_net_unscale": [c_ll, vp, vp, vp, vp, vp],
        "gmg_net_adam": [c_ll, vp, vp, vp, vp, c_int, c_float, c_float, c_float, c_float, vp, vp, c_int, c_int, vp],
        "gmg_net_zero": [c_ll, vp, vp],
    }
    for name, args in sig.items():
        getattr(L, name).argtypes = args


def net_call(name: str, *args) -> None:
    """Call one gmg_net_* entry point; raise on a non-zero status."""
    rc = getattr(lib(), name)(*args)
    if rc != 0:
        raise GmgError(f"{name} failed with status {rc}")


def declared_functions() -> List[str]:
    """Names of the functions declared in include/gmg.h and include/gmg_net.h."""
    names = set()
    for path in (HEADER, NET_HEADER):
        text = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gmg_\w+)\s*\(", text, flags=re.M))
    return sorted(names)


def tune_export() -> str:
    """The autotuner's table (launch shapes per level geometry) as text (gmg_tune_export)."""
    L = lib()
    n = ctypes.c_size_t(0)
    if L.gmg_tune_export(None, 0, ctypes.byref(n)) != OK:
        raise GmgError("gmg_tune_export failed")
    buf = ctypes.create_string_buffer(n.value + 1)
    if L.gmg_tune_export(buf, n.value + 1, ctypes.byref(n)) != OK:
        raise GmgError("gmg_tune_export failed")
    return buf.value.decode()


def tune_import(text: str) -> None:
    """Merge an exported tuning table into this process's (gmg_tune_import)."""
    if lib().gmg_tune_import(text.encode()) != OK:
        raise GmgError("gmg_tune_import: malformed tuning table")


def test_ring_wait_tries(tries: int) -> None:
    """Test hook (gmg_test_ring_wait_tries): poll limit of the pipelined kernels' ring
    waits on the current device; a negative value restores the default."""
    _check(lib().gmg_test_ring_wait_tries(int(tries)), None)


def test_cluster_ranks(ranks: int) -> None:
    """Test hook (gmg_test_cluster_ranks): largest cluster size of the cluster-form
    bottom in handles planned afterwards (16 or 8; 0 restores the default)."""
    _check(lib().gmg_test_cluster_ranks(int(ranks)), None)


def options(coarsen: str = "aniso", precision: str = "fp32", **kw) -> Options:
    o = Options()
    lib().gmg_default_options(ctypes.byref(o))
    o.coarsen = ANISO if coarsen == "aniso" else ISO
    o.precision = PRECISIONS[precision]
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def _ivec(v) -> ctypes.Array:
    return (ctypes.c_int * len(v))(*[int(x) for x in v])


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr(t, dtype=None, numel=None) -> int:
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected dtype {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return t.data_ptr()


def _check(rc: int, handle, batch: bool = False, ok=(OK,)):
    if rc in ok:
        return rc
    L = lib()
    msg = (L.gmg_batch_last_error if batch else L.gmg_last_error)(handle)
    raise GmgError(f"{STATUS_NAMES.get(rc, rc)}: {msg.decode() if msg else ''}")


SOLVE_STATUSES = (OK, NOT_CONVERGED, DIVERGED, NONFINITE)


class Solver:
    """One grid; wraps gmg_create / gmg_set_coeffs / gmg_solve / gmg_destroy."""

    def __init__(self, dims, periodic=(False, False, False), opts: Optional[Options] = None,
                 stream=None, **kw):
        self.dims = tuple(int(d) for d in dims)
        self.periodic = tuple(bool(p) for p in periodic)
        self.opts = opts if opts is not None else options(**kw)
        self.stream = _stream(stream)
        self.h = ctypes.c_void_p()
        rc = lib().gmg_create(ctypes.byref(self.h), *self.dims, _ivec(self.periodic),
                              ctypes.byref(self.opts), ctypes.c_void_p(self.stream))
        _check(rc, None)
        self.ncells = self.dims[0] * self.dims[1] * self.dims[2]
        self.fp64 = self.opts.precision in (IR64, IR64_FP32)

    def close(self):
        if self.h:
            lib().gmg_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_coeffs(self, bx, by, bz):
        import torch
        ptrs = [_ptr(t, torch.float32, self.ncells) for t in (bx, by, bz)]
        _check(lib().gmg_set_coeffs(self.h, *ptrs), self.h)

    def solve(self, sigma, p, tol: float = 1e-6) -> Info:
        """p (in: initial guess, out: solution); returns the Info record."""
        import torch
        dt = torch.float64 if self.fp64 else torch.float32
        info = Info()
        rc = lib().gmg_solve(self.h, _ptr(sigma, dt, self.ncells), _ptr(p, dt, self.ncells),
                             float(tol), ctypes.byref(info))
        _check(rc, self.h, ok=SOLVE_STATUSES)
        return info

    def pcg_solve(self, sigma, p, tol: float = 1e-6, max_iter: int = 10000) -> Info:
        """Jacobi-preconditioned CG on the finest level (gmg_pcg_solve): float32 sigma
        and p (in: initial guess, out: solution); info.cycles = CG iterations."""
        import torch
        info = Info()
        rc = lib().gmg_pcg_solve(self.h, _ptr(sigma, torch.float32, self.ncells), _ptr(p, torch.float32, self.ncells),
                                 float(tol), int(max_iter), ctypes.byref(info))
        _check(rc, self.h, ok=SOLVE_STATUSES)
        return info

    def gmgpcg_solve(self, sigma, p, tol: float = 1e-6) -> Info:
        """Multigrid with PCG as the smoother (gmg_gmgpcg_solve): float32 sigma and p;
        info.cycles = V-cycles."""
        import torch
        info = Info()
        rc = lib().gmg_gmgpcg_solve(self.h, _ptr(sigma, torch.float32, self.ncells),
                                    _ptr(p, torch.float32, self.ncells), float(tol), ctypes.byref(info))
        _check(rc, self.h, ok=SOLVE_STATUSES)
        return info

    def solve_host(self, sigma, p, tol: float = 1e-6) -> Info:
        """As solve, with sigma and p host numpy arrays (or pinned CPU tensors)."""
        import numpy as np
        dt = np.float64 if self.fp64 else np.float32

        def hp(a):
            if hasattr(a, "data_ptr"):
                import torch
                tdt = torch.float64 if self.fp64 else torch.float32
                if a.is_cuda or not a.is_contiguous() or a.numel() != self.ncells:
                    raise ValueError("expected a contiguous CPU tensor of the grid size")
                if a.dtype != tdt:
                    raise ValueError(f"expected a CPU tensor of dtype {tdt}, got {a.dtype}")
                return a.data_ptr()
            if a.dtype != dt or not a.flags.c_contiguous or a.size != self.ncells:
                raise ValueError(f"expected a C-contiguous {dt.__name__} array of the grid size")
            return a.ctypes.data
        info = Info()
        rc = lib().gmg_solve_host(self.h, ctypes.c_void_p(hp(sigma)), ctypes.c_void_p(hp(p)),
                                  float(tol), ctypes.byref(info))
        _check(rc, self.h, ok=SOLVE_STATUSES)
        return info

    def test_poison_omega(self, cycle: int) -> None:
        """Test hook (gmg_test_poison_omega): NaN into the device omega before V-cycle `cycle`
        of the next solve."""
        _check(lib().gmg_test_poison_omega(self.h, int(cycle)), self.h)

    def history(self, cap: int = 1000):
        import numpy as np
        res = np.zeros(cap + 1)
        om = np.zeros(cap)
        acc = np.zeros(cap, dtype=np.int32)
        n = lib().gmg_history(self.h, res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              acc.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), cap)
        if n < 0:
            raise GmgError(lib().gmg_last_error(self.h).decode())
        return res[:n + 1], om[:n], acc[:n].astype(bool)

    def bottom_form(self):
        """(first level of the bottom kernel, CTAs running it: 1 = one CTA, > 1 =
        a thread-block cluster; (0, 0) = no bottom kernel)  (gmg_bottom_form)."""
        lv, rk = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().gmg_bottom_form(self.h, ctypes.byref(lv), ctypes.byref(rk)), self.h)
        return lv.value, rk.value

    def levels(self):
        L = lib().gmg_levels(self.h, None)
        arr = (ctypes.c_int * (3 * L))()
        lib().gmg_levels(self.h, arr)
        return [tuple(arr[3 * l:3 * l + 3]) for l in range(L)]


class BatchSolver:
    """Many independent problems; wraps gmg_batch_*."""

    def __init__(self, dims: Sequence, periodic=None, opts: Optional[Options] = None, stream=None,
                 **kw):
        self.dims = [tuple(int(x) for x in d) for d in dims]
        self.n = len(self.dims)
        self.opts = opts if opts is not None else options(**kw)
        self.stream = _stream(stream)
        flat = _ivec([x for d in self.dims for x in d])
        per = None if periodic is None else _ivec([int(bool(x)) for p in periodic for x in p])
        self.h = ctypes.c_void_p()
        rc = lib().gmg_batch_create(ctypes.byref(self.h), self.n, flat, per, ctypes.byref(self.opts),
                                    ctypes.c_void_p(self.stream))
        _check(rc, None, batch=True)
        self.ncells = [d[0] * d[1] * d[2] for d in self.dims]

    def close(self):
        if self.h:
            lib().gmg_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _arr(self, tensors, dtype):
        if len(tensors) != self.n:
            raise ValueError(f"expected {self.n} tensors")
        return (ctypes.c_void_p * self.n)(*[_ptr(t, dtype, n) for t, n in zip(tensors, self.ncells)])

    def set_coeffs(self, bx, by, bz):
        import torch
        f = torch.float32
        _check(lib().gmg_batch_set_coeffs(self.h, self._arr(bx, f), self._arr(by, f), self._arr(bz, f)),
               self.h, batch=True)

    def solve(self, sigma, p, tol: float = 1e-6) -> List[Info]:
        """sigma, p: lists of device tensors, float32 (or float64 in the FP64 refinement modes)."""
        import torch
        dt = torch.float64 if self.opts.precision in (IR64, IR64_FP32) else torch.float32
        infos = (Info * self.n)()
        rc = lib().gmg_batch_solve(self.h, self._arr(sigma, dt), self._arr(p, dt), float(tol), infos)
        _check(rc, self.h, batch=True, ok=SOLVE_STATUSES)
        return list(infos)


# ---------------------------------------------------------------- single steps

def _dims_of(t):
    nz, ny, nx = t.shape
    return nx, ny, nz


def op_sweep(bx, by, bz, b, p_in, p_out, omega, periodic=(False, False, False), stream=None):
    import torch
    dims = _dims_of(b)
    n = b.numel()
    ptrs = [_ptr(t, torch.float32, n) for t in (bx, by, bz, b, p_in, p_out)]
    rc = lib().gmg_op_sweep(*dims, _ivec(periodic), *ptrs, float(omega), ctypes.c_void_p(_stream(stream)))
    _check(rc, None)


def op_sweep_reference(bx, by, bz, b, p, omega, periodic=(False, False, False), stream=None):
    import torch
    dims = _dims_of(b)
    n = b.numel()
    ptrs = [_ptr(t, torch.float32, n) for t in (bx, by, bz, b, p)]
    rc = lib().gmg_op_sweep_reference(*dims, _ivec(periodic), *ptrs, float(omega),
                                      ctypes.c_void_p(_stream(stream)))
    _check(rc, None)


def op_residual_restrict(bx, by, bz, b, p, b_coarse, factors, periodic=(False, False, False),
                         want_norm: bool = False, stream=None):
    import torch
    dims = _dims_of(b)
    n = b.numel()
    ptrs = [_ptr(t, torch.float32, n) for t in (bx, by, bz, b, p)]
    rr = ctypes.c_double(0.0)
    rc = lib().gmg_op_residual_restrict(*dims, _ivec(periodic), _ivec(factors), *ptrs,
                                        _ptr(b_coarse, torch.float32),
                                        ctypes.byref(rr) if want_norm else None,
                                        ctypes.c_void_p(_stream(stream)))
    _check(rc, None)
    return rr.value if want_norm else None


def op_residual_norm(bx, by, bz, b, p, periodic=(False, False, False), stream=None) -> float:
    import torch
    dims = _dims_of(b)
    n = b.numel()
    ptrs = [_ptr(t, torch.float32, n) for t in (bx, by, bz, b, p)]
    rr = ctypes.c_double(0.0)
    rc = lib().gmg_op_residual_norm(*dims, _ivec(periodic), *ptrs, ctypes.byref(rr),
                                    ctypes.c_void_p(_stream(stream)))
    _check(rc, None)
    return rr.value


def op_residual_norm_noalloc(bx, by, bz, b, p, periodic=(False, False, False), stream=None) -> float:
    """As op_residual_norm, with the library's fixed scratch array (no allocation)."""
    import torch
    dims = _dims_of(b)
    n = b.numel()
    ptrs = [_ptr(t, torch.float32, n) for t in (bx, by, bz, b, p)]
    rr = ctypes.c_double(0.0)
    rc = lib().gmg_op_residual_norm_noalloc(*dims, _ivec(periodic), *ptrs, ctypes.byref(rr),
                                            ctypes.c_void_p(_stream(stream)))
    _check(rc, None)
    return rr.value


def op_residual64(bx, by, bz, b, p, periodic=(False, False, False), definition: int = 0, r_out=None, r32_out=None,
                  stream=None) -> float:
    """r = b - A p of the FP64 refinement (gmg_op_residual64): float64 b and p, float32
    faces; definition 0 (the solver's double-length FP32 evaluation) or 1 (all FP64).
    Writes r into r_out (float64) and/or r32_out (float32); returns sum r32^2."""
    import torch
    dims = _dims_of(b)
    n = b.numel()
    fp = [_ptr(t, torch.float32, n) for t in (bx, by, bz)]
    rr = ctypes.c_double(0.0)
    rc = lib().gmg_op_residual64(*dims, _ivec(periodic), *fp, _ptr(b, torch.float64, n), _ptr(p, torch.float64, n),
                                 _ptr(r_out, torch.float64, n) if r_out is not None else None,
                                 _ptr(r32_out, torch.float32, n) if r32_out is not None else None,
                                 ctypes.byref(rr), int(definition), ctypes.c_void_p(_stream(stream)))
    _check(rc, None)
    return rr.value


def op_prolong_add(e, p, factors, stream=None):
    import torch
    dims = _dims_of(p)
    rc = lib().gmg_op_prolong_add(*dims, _ivec(factors), _ptr(e, torch.float32),
                                  _ptr(p, torch.float32), ctypes.c_void_p(_stream(stream)))
    _check(rc, None)


def op_coarsen_coeffs(bx, by, bz, cbx, cby, cbz, factors, periodic=(False, False, False), stream=None):
    import torch
    dims = _dims_of(bx)
    n = bx.numel()
    ptrs = [_ptr(t, torch.float32, n) for t in (bx, by, bz)]
    cptrs = [_ptr(t, torch.float32) for t in (cbx, cby, cbz)]
    rc = lib().gmg_op_coarsen_coeffs(*dims, _ivec(periodic), _ivec(factors), *ptrs, *cptrs,
                                     ctypes.c_void_p(_stream(stream)))
    _check(rc, None)
