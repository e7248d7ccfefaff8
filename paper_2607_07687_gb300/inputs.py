"""Seeded synthetic inputs for the variable-coefficient pressure Poisson solve.

This module only builds inputs: right-hand sides b and face coefficients
beta on a cell-centred Cartesian grid.  It contains none of the solver's
arithmetic (no operator application, smoothing, transfer or norm) and it
imports nothing from the solver or from the checking code, so both sides
can be fed from it.

Conventions (shared with every caller):

* arrays are C-contiguous with shape ``(nz, ny, nx)``; x is the fastest axis;
* cell ``(i, j, k)`` has its centre at ``(i + 1/2, j + 1/2, k + 1/2)`` in grid
  units (spacing 1);
* ``bx[k, j, i]`` is the coefficient on the lower x-face of cell ``(i, j, k)``,
  located at ``(i, j + 1/2, k + 1/2)``; ``by`` and ``bz`` likewise;
* the right-hand side is returned already multiplied by h^2, i.e. in grid
  units, so the discrete problem is ``sum_faces beta_f (p_nb - p_I) = b_I``.

The workloads follow the paper's two test flows (Sec. 2: a Taylor-Green vortex
in a triple-periodic cube, and flow past a sphere in a (16 x 6 x 6)D channel)
and its immersed-body use case (Sec. 3.1: variable-coefficient Poisson
equations of immersed-boundary flows).  The flows themselves are not
simulated; only fields with their shapes and structure are drawn.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

RAMP_HALF_WIDTH = 2.0  # cells: beta ramps from 0 to 1 over d in [-2, 2]


# ----------------------------------------------------------------------------
# Taylor-Green source (periodic cube)
# ----------------------------------------------------------------------------

def taylor_green_rhs(n: int, seed: int, noise_var: float = 1e-2) -> np.ndarray:
    """b = h^2 (div_h u_TG + noise) on an n^3 triple-periodic grid over [0, 2pi)^3.

    u = sin x cos y cos z, v = -cos x sin y cos z, w = 0 is sampled at the
    face centres; div_h is the staggered difference of face velocities.  The
    sampled field is discretely divergence free up to rounding, so the seeded
    Gaussian noise (variance ``noise_var``) is what carries the problem.
    Returns float64 of shape (n, n, n).
    """
    h = 2.0 * math.pi / n
    face = np.arange(n + 1, dtype=np.float64) * h          # face coordinates
    cent = (np.arange(n, dtype=np.float64) + 0.5) * h      # cell centres
    # u on x-faces: (n_z, n_y, n_x + 1)
    u = (np.sin(face)[None, None, :] * np.cos(cent)[None, :, None]
         * np.cos(cent)[:, None, None])
    # v on y-faces: (n_z, n_y + 1, n_x)
    v = (-np.cos(cent)[None, None, :] * np.sin(face)[None, :, None]
         * np.cos(cent)[:, None, None])
    div = (u[:, :, 1:] - u[:, :, :-1]) + (v[:, 1:, :] - v[:, :-1, :])   # h * div_h
    del u, v
    rng = np.random.default_rng(seed)
    noise = rng.standard_normal((n, n, n)) * math.sqrt(noise_var)
    return h * div + (h * h) * noise


# ----------------------------------------------------------------------------
# Immersed bodies and face coefficients
# ----------------------------------------------------------------------------

@dataclass
class Body:
    kind: str                      # "sphere", "box" or "cylinder" (axis along z)
    center: Tuple[float, float, float]   # (x, y, z) in grid units
    r: float                       # radius (sphere) or half-width (box)


def _signed_distance(body: Body, x, y, z):
    cx, cy, cz = body.center
    if body.kind == "sphere":
        return np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) - body.r
    if body.kind == "box":
        return np.maximum(np.maximum(np.abs(x - cx), np.abs(y - cy)),
                          np.abs(z - cz)) - body.r
    if body.kind == "cylinder":
        return np.sqrt((x - cx) ** 2 + (y - cy) ** 2) + 0.0 * z - body.r
    raise ValueError(f"unknown body kind {body.kind!r}")


def _ramp(d):
    """0 inside (d <= -2), 1 outside (d >= 2), 0.5 (1 + sin(pi d / 4)) between."""
    w = RAMP_HALF_WIDTH
    out = 0.5 * (1.0 + np.sin(np.pi * np.clip(d, -w, w) / (2.0 * w)))
    out = np.where(d <= -w, 0.0, out)
    out = np.where(d >= w, 1.0, out)
    return out


def body_beta(shape: Tuple[int, int, int], bodies: Sequence[Body],
              upper_faces: bool = False):
    """Face coefficients of a flow with immersed bodies (walls not applied).

    ``shape`` is (nz, ny, nx).  Each face gets the minimum over bodies of the
    cosine ramp of its signed distance.  Returns (bx, by, bz), float64, each
    of ``shape``; with ``upper_faces`` each array also holds the faces on the
    upper domain end along its own axis (n + 1 entries on that axis).
    """
    nz, ny, nx = shape
    extra = 1 if upper_faces else 0
    xc = np.arange(nx, dtype=np.float64) + 0.5
    yc = np.arange(ny, dtype=np.float64) + 0.5
    zc = np.arange(nz, dtype=np.float64) + 0.5
    xf = np.arange(nx + extra, dtype=np.float64)
    yf = np.arange(ny + extra, dtype=np.float64)
    zf = np.arange(nz + extra, dtype=np.float64)
    out = []
    for (X, Y, Z) in ((xf, yc, zc), (xc, yf, zc), (xc, yc, zf)):
        Xg = X[None, None, :]
        Yg = Y[None, :, None]
        Zg = Z[:, None, None]
        b = np.ones((len(Z), len(Y), len(X)), dtype=np.float64)
        for body in bodies:
            b = np.minimum(b, _ramp(_signed_distance(body, Xg, Yg, Zg)))
        out.append(np.ascontiguousarray(b))
    return tuple(out)


def apply_walls(bx, by, bz, periodic=(False, False, False)):
    """Return copies with the lower boundary faces of non-periodic axes set to 0."""
    bx, by, bz = bx.copy(), by.copy(), bz.copy()
    if not periodic[0]:
        bx[:, :, 0] = 0.0
    if not periodic[1]:
        by[:, 0, :] = 0.0
    if not periodic[2]:
        bz[0, :, :] = 0.0
    return bx, by, bz


# ----------------------------------------------------------------------------
# Solenoidal velocity and its divergence through the body
# ----------------------------------------------------------------------------

@dataclass
class FourierPotential:
    """A = amp * sum_m a_m cos(2 pi m.x/L + phi_m), per component."""
    waves: np.ndarray      # (3, M, 3) integer wave numbers per component
    coef: np.ndarray       # (3, M)
    phase: np.ndarray      # (3, M)
    amp: float

    @staticmethod
    def draw(rng: np.random.Generator, kmax: int = 4, modes: int = 8,
             amp: float = 0.1) -> "FourierPotential":
        cand = [(a, b, c) for a in range(-kmax, kmax + 1)
                for b in range(-kmax, kmax + 1) for c in range(0, kmax + 1)
                if 0 < a * a + b * b + c * c <= kmax * kmax]
        cand = np.array(cand, dtype=np.int64)
        waves = np.stack([cand[rng.choice(len(cand), modes, replace=False)]
                          for _ in range(3)])
        coef = rng.standard_normal((3, modes)) / math.sqrt(modes)
        phase = rng.uniform(0.0, 2.0 * math.pi, (3, modes))
        return FourierPotential(waves, coef, phase, amp)

    @staticmethod
    def draw_planar(rng: np.random.Generator, kmax: int = 4, modes: int = 8,
                    amp: float = 0.1) -> "FourierPotential":
        """A = (0, 0, A_z(x, y)): a velocity in the x-y plane with no z dependence
        (the 2D flows of the paper's Fig. 2)."""
        cand = [(a, b, 0) for a in range(-kmax, kmax + 1) for b in range(-kmax, kmax + 1)
                if 0 < a * a + b * b <= kmax * kmax]
        cand = np.array(cand, dtype=np.int64)
        waves = np.stack([cand[rng.choice(len(cand), modes, replace=False)] for _ in range(3)])
        coef = rng.standard_normal((3, modes)) / math.sqrt(modes)
        coef[0] = 0.0
        coef[1] = 0.0
        phase = rng.uniform(0.0, 2.0 * math.pi, (3, modes))
        return FourierPotential(waves, coef, phase, amp)

    def curl(self, x, y, z, L):
        """Analytic curl of A at the given points (broadcast arrays)."""
        # dA_c/dx_d for c, d in 0..2
        grad = [[0.0] * 3 for _ in range(3)]
        for c in range(3):
            for m in range(self.waves.shape[1]):
                kv = 2.0 * math.pi * self.waves[c, m] / np.asarray(L, dtype=np.float64)
                arg = kv[0] * x + kv[1] * y + kv[2] * z + self.phase[c, m]
                s = -self.amp * self.coef[c, m] * np.sin(arg)
                for d in range(3):
                    if kv[d] != 0.0:
                        grad[c][d] = grad[c][d] + s * kv[d]
        cx = grad[2][1] - grad[1][2]
        cy = grad[0][2] - grad[2][0]
        cz = grad[1][0] - grad[0][1]
        return cx, cy, cz


@dataclass
class VortexBlobs:
    """A = sum_b Gamma_b e_b exp(-|x - c_b|^2 / (2 s^2)): Gaussian vortex blobs."""
    centers: np.ndarray    # (B, 3) x, y, z
    axes: np.ndarray       # (B, 3) unit vectors
    gamma: np.ndarray      # (B,)
    s: float

    def curl(self, x, y, z, L):
        cx = cy = cz = 0.0
        for c, e, g in zip(self.centers, self.axes, self.gamma):
            dx, dy, dz = x - c[0], y - c[1], z - c[2]
            phi = g * np.exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * self.s ** 2))
            gx, gy, gz = (-dx * phi / self.s ** 2, -dy * phi / self.s ** 2,
                          -dz * phi / self.s ** 2)
            # curl(e * phi) = grad(phi) x e
            cx = cx + (gy * e[2] - gz * e[1])
            cy = cy + (gz * e[0] - gx * e[2])
            cz = cz + (gx * e[1] - gy * e[0])
        return cx, cy, cz


def solenoidal_rhs(shape, bodies, potential, u_inf: float = 1.0):
    """b = div_h(beta_flow * u) with u = u_inf e_x + curl A sampled at faces.

    ``beta_flow`` are the body coefficients without walls, evaluated on every
    face including the two domain ends: the flow passes through the ends, so
    the wall faces carry no artificial source and b is non-zero only where
    beta varies (the body's boundary source) and where the sampled field is
    not discretely solenoidal.  Returns float64 of ``shape``.
    """
    nz, ny, nx = shape
    L = (float(nx), float(ny), float(nz))
    beta = body_beta(shape, bodies, upper_faces=True)
    xc = np.arange(nx, dtype=np.float64) + 0.5
    yc = np.arange(ny, dtype=np.float64) + 0.5
    zc = np.arange(nz, dtype=np.float64) + 0.5
    flux = []
    for axis in range(3):
        X = (np.arange(nx + 1, dtype=np.float64) if axis == 0 else xc)[None, None, :]
        Y = (np.arange(ny + 1, dtype=np.float64) if axis == 1 else yc)[None, :, None]
        Z = (np.arange(nz + 1, dtype=np.float64) if axis == 2 else zc)[:, None, None]
        vel = np.broadcast_to(np.asarray(potential.curl(X, Y, Z, L)[axis], dtype=np.float64),
                              beta[axis].shape).copy()
        if axis == 0:
            vel += u_inf
        flux.append(beta[axis] * vel)
    fx, fy, fz = flux
    return ((fx[:, :, 1:] - fx[:, :, :-1]) + (fy[:, 1:, :] - fy[:, :-1, :])
            + (fz[1:, :, :] - fz[:-1, :, :]))


# ----------------------------------------------------------------------------
# Complete problems
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    shape: Tuple[int, int, int]          # (nz, ny, nx)
    periodic: Tuple[bool, bool, bool]    # (x, y, z)
    b: np.ndarray                        # float64 (nz, ny, nx), grid units
    bx: np.ndarray
    by: np.ndarray
    bz: np.ndarray
    bodies: List[Body] = field(default_factory=list)
    name: str = ""

    @property
    def dims(self):
        nz, ny, nx = self.shape
        return (nx, ny, nz)

    @property
    def cells(self) -> int:
        return int(np.prod(self.shape))


def taylor_green_problem(n: int = 32, seed: int = 0) -> Problem:
    """Triple-periodic n^3 cube, beta = 1 on every face, Taylor-Green source."""
    shape = (n, n, n)
    ones = np.ones(shape, dtype=np.float64)
    return Problem(shape, (True, True, True), taylor_green_rhs(n, seed),
                   ones, ones.copy(), ones.copy(), [], f"taylor_green_{n}^3")


def sphere_channel_problem(nx: int = 256, ny: int = 96, nz: int = 96,
                           seed: int = 1, radius: float = 8.0,
                           center_x: float = 48.0, u_inf: float = 1.0) -> Problem:
    """Sphere in a walled channel, (16 x 6 x 6)D at D = 16 cells by default."""
    shape = (nz, ny, nx)
    bodies = [Body("sphere", (center_x, ny / 2.0, nz / 2.0), radius)]
    rng = np.random.default_rng(seed)
    pot = FourierPotential.draw(rng)
    b = solenoidal_rhs(shape, bodies, pot, u_inf)
    bx, by, bz = apply_walls(*body_beta(shape, bodies))
    return Problem(shape, (False, False, False), b, bx, by, bz, bodies,
                   f"sphere_channel_{nx}x{ny}x{nz}")


def cylinder_channel_problem(nx: int = 256, ny: int = 64, nz: int = 1, seed: int = 5,
                             radius: float = 8.0, center_x: float = 48.0,
                             periodic_z: bool = False, u_inf: float = 1.0) -> Problem:
    """A circular cylinder (axis along z) in a channel walled in x and y.

    nz = 1 is the 2D flow past a circle (planar potential, no z coupling);
    periodic_z gives the spanwise-periodic cylinder, whose velocity varies along
    the span.  The source is the solenoidal-divergence recipe of the sphere
    channel with these bodies and potentials."""
    shape = (nz, ny, nx)
    periodic = (False, False, bool(periodic_z))
    bodies = [Body("cylinder", (center_x, ny / 2.0, nz / 2.0), radius)]
    rng = np.random.default_rng(seed)
    pot = FourierPotential.draw_planar(rng) if nz == 1 else FourierPotential.draw(rng)
    b = solenoidal_rhs(shape, bodies, pot, u_inf)
    bx, by, bz = apply_walls(*body_beta(shape, bodies), periodic=periodic)
    kind = "2d" if nz == 1 else ("spanwise_periodic" if periodic_z else "walled")
    return Problem(shape, periodic, b, bx, by, bz, bodies, f"cylinder_{kind}_{nx}x{ny}x{nz}")


class _NoPotential:
    """A = 0: the uniform stream alone."""

    @staticmethod
    def curl(x, y, z, L):
        return 0.0, 0.0, 0.0


IMPULSIVE_GEOMETRIES = ("cylinder_2d", "cylinder_spanwise", "sphere")


def impulsive_sources(kind: str, nx: int, ny: int = 64, nz: int = None, steps: int = 4, seed: int = 5,
                      radius: float = 8.0, center_x: float = 32.0, u_inf: float = 1.0):
    """Sources of the pressure solves of the first `steps` time steps of an
    impulsive start (the setting of the paper's Fig. 2): the body moves at u_inf
    from t = 0, and every step has a predictor and a corrector projection, i.e.
    2 * steps solves on fixed coefficients.  Solve k (k = 0, 1, ...) has

        b_k = div_h(beta_flow (u_inf e_x + c_k curl A)),   c_k = k / (2 steps),

    with A the geometry's seeded potential (planar for the 2D cylinder): the
    first solve sees the body's source of the uniform stream alone (the
    low-wavenumber axial pressure wave of an impulsive start), and the vortical
    part of the intermediate velocity builds up over the steps.  By linearity
    b_k = b_body + c_k b_vort, both computed once.

    kind: "cylinder_2d" (nz = 1), "cylinder_spanwise" (z periodic, nz = 32 by
    default) or "sphere" (walls, nz = 64 by default).  Returns (problem, [b_0,
    b_1, ...]): the problem carries the coefficients and b_0."""
    if kind not in IMPULSIVE_GEOMETRIES:
        raise ValueError(f"kind must be one of {IMPULSIVE_GEOMETRIES}")
    if nz is None:
        nz = {"cylinder_2d": 1, "cylinder_spanwise": 32, "sphere": 64}[kind]
    shape = (nz, ny, nx)
    if kind == "sphere":
        periodic = (False, False, False)
        bodies = [Body("sphere", (center_x, ny / 2.0, nz / 2.0), radius)]
    else:
        periodic = (False, False, kind == "cylinder_spanwise")
        bodies = [Body("cylinder", (center_x, ny / 2.0, nz / 2.0), radius)]
    rng = np.random.default_rng(seed)
    pot = FourierPotential.draw_planar(rng) if nz == 1 else FourierPotential.draw(rng)
    b_body = solenoidal_rhs(shape, bodies, _NoPotential(), u_inf)
    b_vort = solenoidal_rhs(shape, bodies, pot, 0.0)
    n = 2 * steps
    rhs = [b_body + (k / n) * b_vort for k in range(n)]
    bx, by, bz = apply_walls(*body_beta(shape, bodies), periodic=periodic)
    prob = Problem(shape, periodic, rhs[0], bx, by, bz, bodies, f"impulsive_{kind}_{nx}x{ny}x{nz}")
    return prob, rhs


def random_bodies(rng: np.random.Generator, dims, count: int) -> List[Body]:
    nx, ny, nz = dims
    out = []
    for _ in range(count):
        kind = "sphere" if rng.random() < 0.5 else "box"
        r = float(rng.uniform(4.0, 12.0))
        c = tuple(float(rng.uniform(r + 2.0, n - r - 2.0)) for n in (nx, ny, nz))
        out.append(Body(kind, c, r))
    return out


def batch_problems(count: int = 64, seed: int = 3) -> List[Problem]:
    """Uneven walled problems with 0-3 random spheres/boxes each."""
    rng = np.random.default_rng(seed)
    xs = list(range(32, 193, 16))
    yz = [32, 48, 64]
    out = []
    for p in range(count):
        nx = int(rng.choice(xs))
        ny = int(rng.choice(yz))
        nz = int(rng.choice(yz))
        nb = int(rng.integers(0, 4))
        bodies = random_bodies(rng, (nx, ny, nz), nb)
        shape = (nz, ny, nx)
        pot = FourierPotential.draw(rng)
        b = solenoidal_rhs(shape, bodies, pot, 1.0)
        bx, by, bz = apply_walls(*body_beta(shape, bodies))
        out.append(Problem(shape, (False, False, False), b, bx, by, bz, bodies,
                           f"batch{p}_{nx}x{ny}x{nz}_b{nb}"))
    return out


class VortexSequence:
    """Sphere-in-channel source advected by three Gaussian vortex blobs.

    Step t moves each blob +1 cell in x; a blob leaving the outlet respawns
    at the inlet with a fresh seeded axis, height and strength.
    """

    def __init__(self, nx: int = 192, ny: int = 64, nz: int = 64, seed: int = 4,
                 radius: float = 8.0, center_x: float = 48.0, blobs: int = 3,
                 blob_sigma: float = 6.0, u_inf: float = 1.0):
        self.shape = (nz, ny, nx)
        self.dims = (nx, ny, nz)
        self.bodies = [Body("sphere", (center_x, ny / 2.0, nz / 2.0), radius)]
        self.walls = apply_walls(*body_beta(self.shape, self.bodies))
        self.rng = np.random.default_rng(seed)
        self.s = blob_sigma
        self.u_inf = u_inf
        self.centers = np.zeros((blobs, 3))
        self.axes = np.zeros((blobs, 3))
        self.gamma = np.zeros(blobs)
        for i in range(blobs):
            self._spawn(i, x=float(self.rng.uniform(0.0, nx)))
        self.t = 0

    def _spawn(self, i, x):
        nx, ny, nz = self.dims
        s = self.s
        self.centers[i] = (x, self.rng.uniform(s, ny - s), self.rng.uniform(s, nz - s))
        a = self.rng.standard_normal(3)
        self.axes[i] = a / np.linalg.norm(a)
        self.gamma[i] = self.rng.uniform(0.5, 1.5) * s

    def rhs(self) -> np.ndarray:
        pot = VortexBlobs(self.centers.copy(), self.axes.copy(), self.gamma.copy(), self.s)
        return solenoidal_rhs(self.shape, self.bodies, pot, self.u_inf)

    def advance(self):
        nx = self.dims[0]
        self.centers[:, 0] += 1.0
        for i in range(len(self.gamma)):
            if self.centers[i, 0] > nx + 3.0 * self.s:
                self._spawn(i, x=-3.0 * self.s)
        self.t += 1

    def problem(self) -> Problem:
        bx, by, bz = self.walls
        return Problem(self.shape, (False, False, False), self.rhs(), bx, by, bz,
                       self.bodies, f"vortex_t{self.t}")


def random_small_problem(dims, periodic, seed: int, zero_blocks: bool = True) -> Problem:
    """Tiny problem with random beta in [0, 1] (zero blocks) for dense checks."""
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    rng = np.random.default_rng(seed)
    bx, by, bz = (rng.uniform(0.0, 1.0, shape) for _ in range(3))
    if zero_blocks:
        for b in (bx, by, bz):
            k0, j0, i0 = (int(rng.integers(0, s)) for s in shape)
            b[k0:k0 + 2, j0:j0 + 2, i0:i0 + 2] = 0.0
    bx, by, bz = apply_walls(bx, by, bz, periodic)
    b = rng.standard_normal(shape)
    return Problem(shape, tuple(periodic), b, bx, by, bz, [], f"random_{nx}x{ny}x{nz}")


def _vortex_rhs(job):
    shape, bodies, centers, axes, gamma, sigma, u_inf = job
    return solenoidal_rhs(shape, bodies, VortexBlobs(centers, axes, gamma, sigma), u_inf).astype(np.float32)


def vortex_frames(count: int, workers: int = 1, **kw):
    """Coefficients and the right-hand sides (float32) of `count` consecutive
    steps of VortexSequence(**kw); the sources are computed in a spawn pool
    of `workers` processes when workers > 1."""
    seq = VortexSequence(**kw)
    jobs = []
    for _ in range(count):
        jobs.append((seq.shape, seq.bodies, seq.centers.copy(), seq.axes.copy(), seq.gamma.copy(), seq.s, seq.u_inf))
        seq.advance()
    if workers > 1 and count > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(min(workers, count)) as pool:
            rhs = pool.map(_vortex_rhs, jobs, chunksize=max(1, count // (4 * workers)))
    else:
        rhs = [_vortex_rhs(j) for j in jobs]
    return seq.walls, rhs
