"""Pins of the FP64 conjugate-gradient oracle (the paper's PCG comparison solver)
against facts fixed outside it: the dense operator's diagonal, a dense
least-squares solve, the FFT closed form, conjugacy of the search directions
and finite termination of CG in exact arithmetic."""
import math

import numpy as np
import pytest

from paper_2607_07687_gb300 import inputs as I


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="module")
def P(O):
    from oracle import pcg_oracle
    return pcg_oracle


def _rand(shape, seed, periodic, zero_block=True):
    rng = np.random.default_rng(seed)
    bx, by, bz = (rng.uniform(0.2, 1.0, shape) for _ in range(3))
    if zero_block:
        for b in (bx, by, bz):
            b[0:2, 0:2, 0:2] = 0.0
    b = rng.standard_normal(shape)
    return b, I.apply_walls(bx, by, bz, periodic)


@pytest.mark.parametrize("periodic", [(False, False, False), (True, False, True), (True, True, True)])
def test_jacobi_diagonal_is_the_operator_diagonal(O, P, periodic):
    shape = (4, 5, 6)
    _, (bx, by, bz) = _rand(shape, 3, periodic)
    A = O.dense_operator(bx, by, bz, periodic)
    np.testing.assert_allclose(P.jacobi_diagonal(bx, by, bz, periodic).ravel(), -np.diag(A), rtol=0, atol=1e-14)


@pytest.mark.parametrize("periodic", [(False, False, False), (True, True, False)])
def test_pcg_matches_dense(O, P, periodic):
    shape = (4, 5, 6)
    b, (bx, by, bz) = _rand(shape, 5, periodic)
    res = P.pcg(b, bx, by, bz, periodic, tol=1e-13, f32_inputs=False)
    assert res.status == 0
    act = P.jacobi_diagonal(bx, by, bz, periodic) > 0
    bp = np.where(act, b - b[act].mean(), 0.0)
    ref = O.dense_solve(bp, bx, by, bz, periodic)
    ref = np.where(act, ref - ref[act].mean(), 0.0)
    assert np.linalg.norm(res.x - ref) / np.linalg.norm(ref) < 1e-10
    np.testing.assert_array_equal(res.x[~act], 0.0)


def test_pcg_terminates_within_n_steps(O, P):
    """In exact arithmetic CG ends after at most as many steps as the system has
    distinct eigenvalues; in FP64 a 60-cell problem is solved within a few more."""
    shape = (3, 4, 5)
    b, (bx, by, bz) = _rand(shape, 7, (False, False, False), zero_block=False)
    res = P.pcg(b, bx, by, bz, tol=1e-12, f32_inputs=False)
    assert res.status == 0 and res.iterations <= 60 + 5


def test_directions_are_conjugate(O, P):
    """Successive search directions are B-conjugate (B = -A), which a wrong alpha
    or beta breaks at once."""
    shape = (4, 4, 6)
    b, (bx, by, bz) = _rand(shape, 9, (False, False, False))
    res = P.pcg(b, bx, by, bz, tol=1e-14, max_iter=12, f32_inputs=False, keep_directions=True)
    D = res.directions
    assert len(D) >= 8
    Bd = [-O.apply_A(d, bx, by, bz) for d in D]
    for i in range(len(D)):
        for j in range(i):
            c = abs(float(np.vdot(D[i], Bd[j])))
            scale = math.sqrt(float(np.vdot(D[i], Bd[i])) * float(np.vdot(D[j], Bd[j])))
            assert c <= 1e-8 * scale, (i, j, c / scale)


def test_pcg_matches_fft(O, P):
    """Triple-periodic 16^3 cube, beta = 1 (Jacobi is a scaled identity there),
    against the FFT solution."""
    n = 16
    rng = np.random.default_rng(11)
    b = rng.standard_normal((n, n, n))
    ones = np.ones((n, n, n))
    res = P.pcg(b, ones, ones, ones, (True, True, True), tol=1e-11, f32_inputs=False)
    assert res.status == 0
    ref = O.fft_solve_periodic(b)
    err = np.linalg.norm(res.x - ref) / np.linalg.norm(ref)
    assert err < 3 * n ** 2 / math.pi ** 2 * 1e-11


def test_history_reaches_tolerance_and_iterations_grow_with_n(O, P):
    """The relative residual reaches tol, and the iteration count grows with the
    grid (the weak scaling the paper holds against PCG)."""
    its = []
    for n in (8, 16, 32):
        prob = I.taylor_green_problem(n, 0)
        res = P.pcg_problem(prob, tol=1e-8, f32_inputs=False)
        assert res.status == 0 and res.history[-1] <= 1e-8
        its.append(res.iterations)
    assert its[0] < its[1] < its[2]


# ---------------------------------------------------------------- GMG-PCG (PCG as the smoother)


@pytest.mark.parametrize("dims,periodic,coarsen", [((8, 8, 8), (False, False, False), "iso"),
                                                   ((12, 8, 4), (True, False, False), "aniso")])
def test_gmg_pcg_matches_dense(O, P, dims, periodic, coarsen):
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    b, (bx, by, bz) = _rand(shape, 13, periodic)
    res = P.gmg_pcg_solve(b, bx, by, bz, periodic, tol=1e-11, coarsen=coarsen, n_min=2, f32_inputs=False)
    assert res.status == 0
    act = P.jacobi_diagonal(bx, by, bz, periodic) > 0
    bp = np.where(act, b - b[act].mean(), 0.0)
    ref = O.dense_solve(bp, bx, by, bz, periodic)
    ref = np.where(act, ref - ref[act].mean(), 0.0)
    assert np.linalg.norm(res.x - ref) / np.linalg.norm(ref) < 1e-9
    assert all(h2 < h1 for h1, h2 in zip(res.history, res.history[1:]))


def test_gmg_pcg_two_grid_correction(O, P):
    """Without smoothing, and with the coarse level solved by enough PCG steps,
    one cycle from zero is the textbook two-grid correction P A_c^+ P^T b
    (dense matrices; P = piecewise-constant injection), up to a constant."""
    shape = (4, 4, 8)
    b, (bx, by, bz) = _rand(shape, 17, (False, False, False), zero_block=False)
    b -= b.mean()
    levels = P.hierarchy(bx, by, bz, (False, False, False), "aniso", 2)[:2]
    fac = levels[0][3]
    nzc, nyc, nxc = shape[0] // fac[2], shape[1] // fac[1], shape[2] // fac[0]
    Pm = np.zeros((np.prod(shape), nzc * nyc * nxc))
    for k in range(shape[0]):
        for j in range(shape[1]):
            for i in range(shape[2]):
                Pm[(k * shape[1] + j) * shape[2] + i, ((k // fac[2]) * nyc + j // fac[1]) * nxc + i // fac[0]] = 1.0
    Ac = O.dense_operator(*levels[1][:3])
    ec = np.linalg.lstsq(Ac, Pm.T @ b.ravel(), rcond=None)[0]
    ref = (Pm @ ec).reshape(shape)
    got = P.gmg_pcg_vcycle(np.zeros(shape), b, levels, 0, 0, 0, 200, (False, False, False))
    d = (got - got.mean()) - (ref - ref.mean())
    assert np.linalg.norm(d) / np.linalg.norm(ref - ref.mean()) < 1e-9
