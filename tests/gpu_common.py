"""Shared helpers of the GPU parity tests (CUDA path vs the FP64 oracle)."""
import functools

import numpy as np

from paper_2607_07687_gb300 import inputs as I


def dev():
    import torch
    return torch.device("cuda:0")


def f32(a) -> np.ndarray:
    """The float64 values of the float32 rounding the GPU receives."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def t32(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev())


def t64(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev())


def host(t) -> np.ndarray:
    return t.detach().cpu().numpy().astype(np.float64)


def rel_l2(a, b) -> float:
    d = np.linalg.norm(np.asarray(a) - np.asarray(b))
    n = np.linalg.norm(np.asarray(b))
    return float(d / n) if n > 0 else float(d)


def gpu_solve(prob, tol, p0=None, **opt):
    """Solve through the C ABI; returns (p float64, info, (history, omegas, accepted))."""
    import torch
    from paper_2607_07687_gb300 import binding as G
    s = G.Solver(prob.dims, prob.periodic, **opt)
    try:
        s.set_coeffs(t32(prob.bx), t32(prob.by), t32(prob.bz))
        if s.fp64:
            b = t64(f32(prob.b))
            p = t64(np.zeros(prob.shape) if p0 is None else p0)
        else:
            b = t32(prob.b)
            p = t32(np.zeros(prob.shape) if p0 is None else p0)
        info = s.solve(b, p, tol)
        torch.cuda.synchronize()
        hist = s.history()
        return host(p), info, hist
    finally:
        s.close()


@functools.lru_cache(maxsize=None)
def oracle_cached(key, tol, **kw):
    from oracle import oracle as O
    prob = problem(key)
    return O.solve_problem(prob, tol=tol, **kw)


@functools.lru_cache(maxsize=None)
def problem(key):
    name, args = key[0], key[1:]
    if name == "tg":
        return I.taylor_green_problem(*args)
    if name == "sphere":
        return I.sphere_channel_problem(*args)
    if name == "cyl":
        return I.cylinder_channel_problem(*args)
    raise KeyError(name)


def random_fields(dims, periodic, seed, zero_blocks=True):
    """Random coefficients in [0, 1] (optionally with zero blocks), right-hand
    side and iterate.  Wall faces are left random: both sides must ignore them."""
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    rng = np.random.default_rng(seed)
    beta = [rng.uniform(0.0, 1.0, shape) for _ in range(3)]
    if zero_blocks:
        for b in beta:
            k0, j0, i0 = (int(rng.integers(0, s)) for s in shape)
            b[k0:k0 + 3, j0:j0 + 3, i0:i0 + 3] = 0.0
    b = rng.standard_normal(shape)
    p = rng.standard_normal(shape)
    return [f32(a) for a in beta], f32(b), f32(p)
