"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks one oracle function against something it does not compute
itself: a hand-worked example, a closed form (Fourier eigenvalues, FFT exact
solution, the smooth Taylor-Green pressure), an independent assembly of the
problem (face-by-face dense matrix, Galerkin triple product), textbook
Gauss-Seidel on that matrix, a dense least-squares solve, or an invariant the
paper states (monotone residual decay under the adaptive relaxation, Sec. 3.1;
fewer V-cycles with anisotropic coarsening, Sec. 3.2).
"""
import math
import os

import numpy as np
import pytest

from paper_2607_07687_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_beta(shape, rng, periodic, zero_block=True):
    bx, by, bz = (rng.uniform(0.0, 1.0, shape) for _ in range(3))
    if zero_block:
        for b in (bx, by, bz):
            k0, j0, i0 = (int(rng.integers(0, s)) for s in shape)
            b[k0:k0 + 2, j0:j0 + 2, i0:i0 + 2] = 0.0
    return I.apply_walls(bx, by, bz, periodic)


def _active(A):
    return np.diag(A) < 0


def _components(A):
    import scipy.sparse.csgraph as cg
    import scipy.sparse as sp
    act = _active(A)
    adj = sp.csr_matrix((A != 0) & ~np.eye(len(A), dtype=bool))
    n, lab = cg.connected_components(adj, directed=False)
    return len(set(lab[act].tolist()))


# ---------------------------------------------------------------- operator


def _read_cases():
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "operator_worked_examples.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = {"dims": tuple(map(int, tok[1:4])), "per": tuple(int(t) != 0 for t in tok[4:7])}
                cases.append(cur)
            else:
                cur[tok[0]] = np.array(list(map(float, tok[1:])))
    return cases


def test_operator_worked_examples(oracle):
    cases = _read_cases()
    assert len(cases) == 3
    for c in cases:
        nx, ny, nz = c["dims"]
        shp = (nz, ny, nx)
        got = oracle.apply_A(c["p"].reshape(shp), c["bx"].reshape(shp), c["by"].reshape(shp),
                             c["bz"].reshape(shp), c["per"])
        np.testing.assert_allclose(got.ravel(), c["Ap"], rtol=0, atol=1e-13)


@pytest.mark.parametrize("dims", [(8, 6, 4), (6, 10, 8), (4, 4, 12)])
def test_operator_fourier_eigenvalues(oracle, dims):
    """Periodic, beta = 1: every Fourier mode is an eigenvector with
    lambda(k) = -sum_d 4 sin^2(pi k_d / n_d)."""
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    ones = np.ones(shape)
    rng = np.random.default_rng(7)
    z, y, x = np.meshgrid(np.arange(nz) + 0.5, np.arange(ny) + 0.5, np.arange(nx) + 0.5, indexing="ij")
    for _ in range(6):
        k = [int(rng.integers(0, n)) for n in dims]
        phase = rng.uniform(0, 2 * math.pi)
        p = np.cos(2 * math.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / nz) + phase)
        lam = -sum(4 * math.sin(math.pi * kd / n) ** 2 for kd, n in zip(k, dims))
        Ap = oracle.apply_A(p, ones, ones, ones, (True, True, True))
        np.testing.assert_allclose(Ap, lam * p, atol=1e-12)


@pytest.mark.parametrize("periodic", [(False, False, False), (True, False, True), (True, True, True)])
def test_operator_matches_face_assembly(oracle, periodic):
    """Cell-by-cell oracle operator == face-by-face dense assembly; the
    assembled matrix is symmetric, annihilates constants and is NSD."""
    shape = (4, 6, 4)
    rng = np.random.default_rng(11)
    bx, by, bz = _rand_beta(shape, rng, periodic)
    A = oracle.dense_operator(bx, by, bz, periodic)
    p = rng.standard_normal(shape)
    np.testing.assert_allclose(oracle.apply_A(p, bx, by, bz, periodic).ravel(), A @ p.ravel(),
                               atol=1e-13)
    np.testing.assert_allclose(A, A.T, atol=0)
    np.testing.assert_allclose(oracle.apply_A(np.ones(shape), bx, by, bz, periodic), 0, atol=1e-14)
    assert np.linalg.eigvalsh(A).max() < 1e-12


def test_operator_energy_identity(oracle):
    """-<p, A p> = sum over faces beta_f (p_P - p_Q)^2, summed face by face."""
    periodic = (False, True, False)
    shape = (5, 4, 6)
    rng = np.random.default_rng(3)
    bx, by, bz = _rand_beta(shape, rng, periodic)
    p = rng.standard_normal(shape)
    energy = 0.0
    for axis, beta in ((2, bx), (1, by), (0, bz)):
        lower = np.roll(p, 1, axis=axis)
        diff2 = (p - lower) ** 2
        if not periodic[2 - axis]:
            sl = [slice(None)] * 3
            sl[axis] = 0
            diff2[tuple(sl)] = 0.0
        energy += float(np.sum(beta * diff2))
    got = -float(np.sum(p * oracle.apply_A(p, bx, by, bz, periodic)))
    assert got == pytest.approx(energy, rel=1e-12)


# ---------------------------------------------------------------- smoother


@pytest.mark.parametrize("periodic", [(False, False, False), (True, True, False)])
def test_half_sweep_zeroes_its_colour(oracle, periodic):
    """omega = 1: after the red half-sweep the residual vanishes on active red
    cells; after the full sweep it vanishes on active black cells."""
    shape = (4, 6, 8)
    rng = np.random.default_rng(5)
    bx, by, bz = _rand_beta(shape, rng, periodic)
    b = rng.standard_normal(shape)
    p = rng.standard_normal(shape)
    k, j, i = np.indices(shape)
    red = (i + j + k) % 2 == 0
    A = oracle.dense_operator(bx, by, bz, periodic)
    act = _active(A).reshape(shape)
    p1 = oracle.half_sweep(p, b, bx, by, bz, 1.0, 0, periodic)
    r1 = b - oracle.apply_A(p1, bx, by, bz, periodic)
    assert np.abs(r1[red & act]).max() < 1e-12
    assert np.abs(r1[red & act]).max() < 1e-6 * np.abs(r1[~red & act]).max()
    np.testing.assert_array_equal(p1[~red], p[~red])
    np.testing.assert_array_equal(p1[~act], p[~act])
    p2 = oracle.sweep(p, b, bx, by, bz, 1.0, periodic)
    r2 = b - oracle.apply_A(p2, bx, by, bz, periodic)
    assert np.abs(r2[~red & act]).max() < 1e-12


@pytest.mark.parametrize("omega", [1.0, 0.6, 1.3])
def test_sweep_equals_textbook_gauss_seidel(oracle, omega):
    """One sweep == textbook SOR on the assembled matrix, red cells first."""
    periodic = (True, False, False)
    shape = (3, 4, 6)
    rng = np.random.default_rng(9)
    bx, by, bz = _rand_beta(shape, rng, periodic)
    b = rng.standard_normal(shape)
    p = rng.standard_normal(shape)
    A = oracle.dense_operator(bx, by, bz, periodic)
    x = p.ravel().copy()
    k, j, i = np.indices(shape)
    colour = ((i + j + k) % 2).ravel()
    for c in (0, 1):
        for n in np.nonzero(colour == c)[0]:
            if A[n, n] == 0:
                continue
            gs = (b.ravel()[n] - (A[n] @ x - A[n, n] * x[n])) / A[n, n]
            x[n] = (1 - omega) * x[n] + omega * gs
    got = oracle.sweep(p, b, bx, by, bz, omega, periodic)
    np.testing.assert_allclose(got.ravel(), x, atol=1e-12)


# ---------------------------------------------------------------- hierarchy


def test_schedule_reading():
    """Coarsening schedules of the workload shapes (Sec. 3.2, reading C3)."""
    from oracle import oracle as O
    d, f = O.schedule((256, 96, 96), coarsen="aniso")
    assert d == [(256, 96, 96), (128, 48, 48), (64, 24, 24), (32, 12, 12), (16, 6, 6),
                 (8, 6, 6), (4, 6, 6)]
    assert f[4] == (2, 1, 1) and f[-1] == (1, 1, 1)
    d, f = O.schedule((256, 96, 96), coarsen="iso")
    assert d == [(256, 96, 96), (128, 48, 48), (64, 24, 24), (32, 12, 12), (16, 6, 6)]
    d, _ = O.schedule((32, 32, 32), (True, True, True), coarsen="iso")
    assert d == [(32, 32, 32), (16, 16, 16), (8, 8, 8), (4, 4, 4)]
    # periodic axes never coarsen to an odd length
    d, _ = O.schedule((40, 8, 8), (True, True, True), coarsen="aniso")
    assert all(n % 2 == 0 for lv in d for n in lv)
    assert d[-1][0] == 10
    # the smallest dimension limits isotropic depth
    d, _ = O.schedule((8, 64, 64), coarsen="iso")
    assert len(d) == 2


def test_schedule_2d():
    """A length-1 axis (the 2D flows of Fig. 2) never halves and does not stop
    isotropic coarsening of the other two (reading C3, singleton axes)."""
    from oracle import oracle as O
    d, f = O.schedule((256, 64, 1), coarsen="iso")
    assert d == [(256, 64, 1), (128, 32, 1), (64, 16, 1), (32, 8, 1), (16, 4, 1)]
    assert all(c[2] == 1 for c in f)
    d, _ = O.schedule((256, 64, 1), coarsen="aniso")
    assert d == [(256, 64, 1), (128, 32, 1), (64, 16, 1), (32, 8, 1), (16, 4, 1), (8, 4, 1), (4, 4, 1)]
    d, _ = O.schedule((1, 1, 1), coarsen="iso")
    assert d == [(1, 1, 1)]


def test_coarse_beta_constant(oracle):
    """beta = 1 coarsens to prod_{e != d} c_e / c_d, the anisotropically spaced
    7-point operator; Neumann wall faces stay zero."""
    shape = (8, 12, 16)
    ones = I.apply_walls(np.ones(shape), np.ones(shape), np.ones(shape))
    for fac in [(2, 2, 2), (2, 1, 1), (1, 2, 2), (2, 1, 2)]:
        cb = oracle.coarsen_beta(*ones, fac)
        for d, c in enumerate(cb):
            expect = np.prod([fac[e] for e in range(3) if e != d]) / fac[d]
            inner = [slice(None)] * 3
            inner[2 - d] = slice(1, None)
            np.testing.assert_allclose(c[tuple(inner)], expect)
            wall = [slice(None)] * 3
            wall[2 - d] = 0
            np.testing.assert_array_equal(c[tuple(wall)], 0.0)


def _prolongation(fine_shape, fac):
    nz, ny, nx = fine_shape
    cz, cy, cx = nz // fac[2], ny // fac[1], nx // fac[0]
    P = np.zeros((nx * ny * nz, cx * cy * cz))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                P[(k * ny + j) * nx + i, ((k // fac[2]) * cy + j // fac[1]) * cx + i // fac[0]] = 1
    return P


@pytest.mark.parametrize("fac", [(2, 2, 2), (2, 1, 1), (1, 2, 2), (2, 1, 2), (1, 2, 1), (1, 1, 2)])
def test_transfers_and_galerkin(oracle, fac):
    """Restriction is the transpose of the piecewise-constant prolongation,
    the finite-volume coarse faces are 1/c_d times the Galerkin ones, and the
    Galerkin option's coarse faces give R A P itself (built by matrix products)."""
    periodic = (False, True, False)
    shape = (4, 4, 8)
    rng = np.random.default_rng(2)
    bx, by, bz = _rand_beta(shape, rng, periodic, zero_block=False)
    P = _prolongation(shape, fac)
    r = rng.standard_normal(shape)
    cshape = (shape[0] // fac[2], shape[1] // fac[1], shape[2] // fac[0])
    e = rng.standard_normal(cshape)
    np.testing.assert_allclose(oracle.restrict(r, fac).ravel(), P.T @ r.ravel(), atol=1e-13)
    np.testing.assert_allclose(oracle.prolong_add(np.zeros(shape), e, fac).ravel(), P @ e.ravel(),
                               atol=0)
    A = oracle.dense_operator(bx, by, bz, periodic)
    RAP = P.T @ A @ P
    cb = oracle.coarsen_beta(bx, by, bz, fac, periodic)
    scaled = [cb[d] * fac[d] for d in range(3)]
    np.testing.assert_allclose(oracle.dense_operator(*scaled, periodic), RAP, atol=1e-12)
    gal = oracle.coarsen_beta(bx, by, bz, fac, periodic, galerkin=True)
    np.testing.assert_allclose(oracle.dense_operator(*gal, periodic), RAP, atol=1e-12)


def _sor_colours(A, b, x, omega, shape):
    k, j, i = np.indices(shape)
    colour = ((i + j + k) % 2).ravel()
    for c in (0, 1):
        for n in np.nonzero(colour == c)[0]:
            if A[n, n] == 0:
                continue
            gs = (b[n] - (A[n] @ x - A[n, n] * x[n])) / A[n, n]
            x[n] = (1 - omega) * x[n] + omega * gs
    return x


def _matrix_vcycle(lv, l, b, x, omega, nu1, nu2, nu_c, dense=False):
    """The V-cycle of Sec. 3 written with dense matrices: smoother, residual,
    R = P^T, recursion, P e, smoother; the coarsest right-hand side is
    projected to zero mean over active cells before its sweeps (or, dense,
    solved by scipy's SVD pseudo-inverse)."""
    import scipy.linalg
    A, shape = lv[l]["A"], lv[l]["shape"]
    if l == len(lv) - 1:
        act = np.diag(A) < 0
        b = np.where(act, b - b[act].mean(), 0.0)
        if dense:
            return scipy.linalg.pinv(A) @ b
        for _ in range(nu_c):
            x = _sor_colours(A, b, x, omega, shape)
        return x
    for _ in range(nu1):
        x = _sor_colours(A, b, x, omega, shape)
    P = lv[l]["P"]
    e = _matrix_vcycle(lv, l + 1, P.T @ (b - A @ x), np.zeros(P.shape[1]), omega, nu1, nu2, nu_c, dense)
    x = x + P @ e
    for _ in range(nu2):
        x = _sor_colours(A, b, x, omega, shape)
    return x


@pytest.mark.parametrize("dims,periodic,coarsen", [((8, 4, 6), (False, False, False), "aniso"),
                                                   ((8, 8, 4), (True, False, True), "aniso"),
                                                   ((8, 8, 8), (False, True, False), "iso")])
def test_vcycle_matches_matrix_form(oracle, dims, periodic, coarsen):
    """One oracle V-cycle from a random iterate and an incompatible right-hand
    side equals the matrix-form V-cycle on the same hierarchy."""
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    rng = np.random.default_rng(31)
    bx, by, bz = _rand_beta(shape, rng, periodic)
    b = rng.standard_normal(shape) + 0.3
    p = rng.standard_normal(shape)
    levels, facs = oracle.schedule(dims, periodic, coarsen=coarsen, n_min=2)
    assert len(levels) >= 3
    lv, beta = [], (bx, by, bz)
    for l, (d, f) in enumerate(zip(levels, facs)):
        sh = (d[2], d[1], d[0])
        entry = {"A": oracle.dense_operator(*beta, periodic), "shape": sh}
        if l + 1 < len(levels):
            entry["P"] = _prolongation(sh, f)
            beta = oracle.coarsen_beta(*beta, f, periodic)
        lv.append(entry)
    omega = 0.8
    ref = _matrix_vcycle(lv, 0, b.ravel(), p.ravel().copy(), omega, 2, 2, 16)
    got = oracle.vcycle(p, b, bx, by, bz, omega, periodic, coarsen=coarsen, n_min=2)
    np.testing.assert_allclose(got.ravel(), ref, rtol=1e-11, atol=1e-11)
    # the dense coarsest solve (coarse_mode 1) in place of the coarsest sweeps
    ref = _matrix_vcycle(lv, 0, b.ravel(), p.ravel().copy(), omega, 2, 2, 16, dense=True)
    got = oracle.vcycle(p, b, bx, by, bz, omega, periodic, coarsen=coarsen, n_min=2, coarse_mode=1)
    np.testing.assert_allclose(got.ravel(), ref, rtol=1e-9, atol=1e-9)
    # the Galerkin option (coarse_op 1): every coarse operator is P^T A P of the
    # level above, formed here by matrix products alone
    glv = [dict(lv[0])]
    for l in range(1, len(lv)):
        P = lv[l - 1]["P"]
        glv.append(dict(lv[l], A=P.T @ glv[l - 1]["A"] @ P))
        glv[l - 1] = dict(glv[l - 1], P=P)
    ref = _matrix_vcycle(glv, 0, b.ravel(), p.ravel().copy(), omega, 2, 2, 16)
    got = oracle.vcycle(p, b, bx, by, bz, omega, periodic, coarsen=coarsen, n_min=2, coarse_op=1)
    np.testing.assert_allclose(got.ravel(), ref, rtol=1e-11, atol=1e-11)


# ---------------------------------------------------------------- dense coarsest solve (option)


@pytest.mark.parametrize("dims,periodic,split", [((4, 6, 6), (False, False, False), False),
                                                 ((4, 6, 6), (False, False, False), True),
                                                 ((4, 4, 4), (True, True, True), False),
                                                 ((6, 4, 4), (True, False, True), True),
                                                 ((8, 6, 1), (False, False, False), False)])
def test_pinv_apply_is_the_minimum_norm_solution(oracle, dims, periodic, split):
    """The coarsest-level step of coarse_mode 1, p = A^+ b from the Jacobi
    eigendecomposition, equals scipy's SVD pseudo-inverse of the face-by-face
    dense assembly applied to b and the gelsd least-squares solve, on an
    incompatible right-hand side: walled, periodic and mixed grids, coefficients
    with zero blocks (isolated cells), and with a zero wall of faces splitting the
    cells into two components (one null vector each)."""
    import scipy.linalg
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    rng = np.random.default_rng(sum(dims) + 3 * split)
    bx, by, bz = _rand_beta(shape, rng, periodic)
    if split:                                   # no face across x = nx / 2 (or wrap): two components
        bx[:, :, nx // 2] = 0.0
        if periodic[0]:
            bx[:, :, 0] = 0.0
    A = oracle.dense_operator(bx, by, bz, periodic)
    assert (_components(A) >= 2) == split
    b = rng.standard_normal(shape) + 0.5
    got = oracle.pinv_apply(b, bx, by, bz, periodic)
    # singular values below 1e-10 of the largest are the null space (rounding level ~1e-15)
    ref = (scipy.linalg.pinv(A, rtol=1e-10) @ b.ravel()).reshape(shape)
    np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-10 * np.abs(ref).max())
    lsq = scipy.linalg.lstsq(A, b.ravel(), cond=1e-10, lapack_driver="gelsd")[0].reshape(shape)
    np.testing.assert_allclose(got, lsq, atol=1e-9 * np.abs(ref).max())
    # minimum norm: orthogonal to the constant vector of every component
    assert abs(got[_active(A).reshape(shape)].sum()) <= 1e-9 * np.abs(got).sum()


def test_pinv_apply_periodic_fft(oracle):
    """beta = 1 on a triple-periodic grid: A^+ b is the FFT closed form of the
    zero-mean part of b."""
    shape = (4, 4, 8)
    rng = np.random.default_rng(9)
    b = rng.standard_normal(shape)
    ones = np.ones(shape)
    got = oracle.pinv_apply(b, ones, ones, ones, (True, True, True))
    np.testing.assert_allclose(got, oracle.fft_solve_periodic(b), atol=1e-11)


@pytest.mark.parametrize("dims,periodic,coarsen", [((8, 8, 8), (False, False, False), "aniso"),
                                                   ((8, 4, 6), (True, False, False), "iso"),
                                                   ((12, 8, 1), (False, False, False), "aniso")])
def test_dense_coarse_solve_matches_dense(oracle, dims, periodic, coarsen):
    """Whole solves with the dense coarsest level converge to the dense
    minimum-norm solution, in fewer V-cycles than with the 16 coarsest sweeps."""
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    rng = np.random.default_rng(sum(dims) + 5)
    bx, by, bz = _rand_beta(shape, rng, periodic)
    A = oracle.dense_operator(bx, by, bz, periodic)
    act = _active(A).reshape(shape)
    b = rng.standard_normal(shape)
    res = oracle.solve(b, bx, by, bz, periodic, tol=1e-12, coarsen=coarsen, max_cycles=400, coarse_mode=1)
    assert res.status == oracle.OK
    bp = np.where(act, b - b[act].mean(), 0.0)
    p_ref = oracle.dense_solve(bp, bx, by, bz, periodic)
    p_ref = np.where(act, p_ref - p_ref[act].mean(), 0.0)
    np.testing.assert_allclose(res.p, p_ref, atol=1e-9 * np.abs(p_ref).max())
    sweeps = oracle.solve(b, bx, by, bz, periodic, tol=1e-12, coarsen=coarsen, max_cycles=400)
    assert res.cycles <= sweeps.cycles, (res.cycles, sweeps.cycles)


# ---------------------------------------------------------------- closed forms


def test_fft_solution_is_exact(oracle):
    """The FFT closed form agrees with a dense least-squares solve."""
    shape = (4, 6, 4)
    rng = np.random.default_rng(4)
    b = rng.standard_normal(shape)
    ones = np.ones(shape)
    p_fft = oracle.fft_solve_periodic(b)
    p_dense = oracle.dense_solve(b - b.mean(), ones, ones, ones, (True, True, True))
    np.testing.assert_allclose(p_fft, p_dense, atol=1e-11)


@pytest.mark.parametrize("dims,periodic", [((8, 8, 8), (False, False, False)),
                                           ((8, 4, 6), (True, False, False)),
                                           ((6, 8, 4), (True, True, True)),
                                           ((5, 7, 4), (False, False, False)),
                                           ((12, 8, 1), (False, False, False)),
                                           ((8, 8, 1), (True, True, False))])
@pytest.mark.parametrize("coarsen", ["iso", "aniso"])
def test_solve_matches_dense(oracle, dims, periodic, coarsen):
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    rng = np.random.default_rng(sum(dims) + 17 * sum(periodic))
    bx, by, bz = _rand_beta(shape, rng, periodic)
    A = oracle.dense_operator(bx, by, bz, periodic)
    assert _components(A) == 1
    act = _active(A).reshape(shape)
    b = rng.standard_normal(shape)
    res = oracle.solve(b, bx, by, bz, periodic, tol=1e-12, coarsen=coarsen, max_cycles=400,
                       n_min=2)
    assert res.status == oracle.OK
    bp = np.where(act, b - b[act].mean(), 0.0)
    p_ref = oracle.dense_solve(bp, bx, by, bz, periodic)
    p_ref = np.where(act, p_ref - p_ref[act].mean(), 0.0)
    err = np.linalg.norm(res.p - p_ref) / np.linalg.norm(p_ref)
    assert err < 1e-9
    np.testing.assert_array_equal(res.p[~act], 0.0)


def test_solve_matches_fft_32(oracle):
    """Taylor-Green cube (32^3, beta = 1, periodic) against the FFT solution."""
    prob = I.taylor_green_problem(32, 0)
    res = oracle.solve_problem(prob, tol=1e-10, coarsen="iso", f32_inputs=False)
    assert res.status == oracle.OK and res.levels == 4
    p_ref = oracle.fft_solve_periodic(prob.b)
    err = np.linalg.norm(res.p - p_ref) / np.linalg.norm(p_ref)
    # relative error <= condition number x relative residual
    assert err < 3 * 32 ** 2 / math.pi ** 2 * 1e-10
    assert err < 1e-9


def test_solve_matches_fft_2d(oracle):
    """A 2D periodic square (64 x 64 x 1, beta = 1) against the FFT solution: the
    length-1 axis has no neighbours, so its Fourier factor is 0."""
    shape = (1, 64, 64)
    rng = np.random.default_rng(8)
    b = rng.standard_normal(shape)
    b -= b.mean()
    ones = np.ones(shape)
    bx, by, bz = I.apply_walls(ones, ones, ones, (True, True, False))
    assert not bz.any()
    res = oracle.solve(b, bx, by, bz, (True, True, False), tol=1e-10, coarsen="iso")
    assert res.status == oracle.OK and res.levels == 5
    p_ref = oracle.fft_solve_periodic(b)
    err = np.linalg.norm(res.p - p_ref) / np.linalg.norm(p_ref)
    assert err < 2 * 64 ** 2 / math.pi ** 2 * 1e-10


def test_smooth_taylor_green_pressure(oracle):
    """b = A_h p for p = (cos 2x + cos 2y)(cos 2z + 2)/16 at cell centres,
    built from the exact eigenvalue -4 sin^2(h) of cos 2x; the solve returns
    p minus its mean."""
    n = 32
    h = 2 * math.pi / n
    c = (np.arange(n) + 0.5) * h
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    lam = -4 * math.sin(h) ** 2
    p_exact = (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2) / 16
    b = lam / 16 * ((np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2)
                    + (np.cos(2 * x) + np.cos(2 * y)) * np.cos(2 * z))
    ones = np.ones_like(b)
    res = oracle.solve(b, ones, ones, ones, (True, True, True), tol=1e-11, coarsen="iso")
    ref = p_exact - p_exact.mean()
    assert np.linalg.norm(res.p - ref) / np.linalg.norm(ref) < 1e-9


# ---------------------------------------------------------------- control


def test_history_monotone_heterogeneous(oracle):
    """Sec. 3.1: the adaptive relaxation keeps the residual non-increasing."""
    prob = I.sphere_channel_problem(64, 32, 32, seed=5, radius=6.0, center_x=20.0)
    res = oracle.solve_problem(prob, tol=1e-8, max_cycles=80)
    assert res.status == oracle.OK
    assert np.all(np.diff(res.history) <= 0)


def test_galerkin_option_solves_with_monotone_history(oracle):
    """C4's Galerkin option (coarse_op 1) on a heterogeneous channel: the
    solve reaches the tolerance with the non-increasing history of Sec. 3.1,
    and its answer agrees with the finite-volume hierarchy's to the tolerance
    (the coarse operator changes the iteration, not the solution)."""
    prob = I.sphere_channel_problem(64, 32, 32, seed=5, radius=6.0, center_x=20.0)
    fv = oracle.solve_problem(prob, tol=1e-9, max_cycles=200)
    gal = oracle.solve_problem(prob, tol=1e-9, max_cycles=200, coarse_op=1)
    assert fv.status == oracle.OK and gal.status == oracle.OK
    assert np.all(np.diff(gal.history) <= 0)
    assert np.linalg.norm(gal.p - fv.p) <= 1e-6 * np.linalg.norm(fv.p)


def test_omega_rejects_growth_then_recovers(oracle):
    """Start over-relaxed (omega0 = 2.4, where SOR amplifies); growing cycles
    are rejected with the iterate kept, omega shrinks by 0.7 each time, and
    the solve still converges with a monotone history."""
    prob = I.sphere_channel_problem(32, 16, 16, seed=6, radius=4.0, center_x=12.0)
    res = oracle.solve_problem(prob, tol=1e-6, omega0=2.4, max_cycles=80)
    assert res.status == oracle.OK
    assert (~res.accepted).sum() >= 1
    assert np.all(np.diff(res.history) <= 0)
    om = res.omegas
    for k in range(len(om) - 1):
        if not res.accepted[k]:
            assert om[k + 1] == pytest.approx(max(0.25, 0.7 * om[k]))
        else:
            assert om[k + 1] == pytest.approx(min(1.0, 1.1 * om[k]))


def test_divergence_reported(oracle):
    """A growing cycle at omega_min ends the solve as diverged and returns the
    last accepted iterate (here the zero guess)."""
    prob = I.sphere_channel_problem(32, 16, 16, seed=6, radius=4.0, center_x=12.0)
    res = oracle.solve_problem(prob, tol=1e-6, omega0=2.6, omega_min=2.6, max_cycles=10)
    assert res.status == oracle.DIVERGED
    assert res.cycles == 1 and not res.accepted[0]
    np.testing.assert_array_equal(res.p, 0.0)


def test_zero_rhs(oracle):
    shape = (8, 8, 8)
    z = np.zeros(shape)
    ones = np.ones(shape)
    res = oracle.solve(z, ones, ones, ones, (True, True, True), tol=1e-6)
    assert res.status == oracle.OK and res.cycles == 0
    np.testing.assert_array_equal(res.p, 0.0)


@pytest.mark.slow
def test_aniso_fewer_cycles_than_iso(oracle):
    """Sec. 3.2: on an elongated channel anisotropic coarsening needs fewer
    V-cycles than isotropic coarsening (aspect ratio 4: 128 x 32 x 32)."""
    prob = I.sphere_channel_problem(128, 32, 32, seed=8, radius=6.0, center_x=24.0)
    iso = oracle.solve_problem(prob, tol=1e-6, coarsen="iso", max_cycles=200)
    ani = oracle.solve_problem(prob, tol=1e-6, coarsen="aniso", max_cycles=200)
    assert iso.status == oracle.OK and ani.status == oracle.OK
    assert ani.cycles < iso.cycles
