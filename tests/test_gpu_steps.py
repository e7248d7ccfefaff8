"""Single multigrid steps on the GPU (through the C ABI) against the oracle,
element by element, on grids spanning several tiles with ragged tails,
periodic and walled axes, and coefficient blocks that vanish."""
import numpy as np
import pytest

from tests.gpu_common import f32, host, random_fields, t32

pytestmark = pytest.mark.gpu

CASES = [((70, 19, 13), (0, 0, 0)), ((66, 18, 14), (1, 1, 1)), ((70, 18, 13), (0, 1, 0)),
         ((33, 9, 2), (0, 0, 0)), ((1, 12, 40), (0, 0, 1)), ((32, 8, 8), (1, 0, 0)),
         ((5, 3, 1), (0, 0, 0)), ((130, 40, 24), (0, 0, 0)), ((2, 4, 6), (1, 1, 1)),
         ((8, 2, 4), (1, 1, 0)), ((64, 16, 9), (0, 0, 0)), ((36, 10, 6), (1, 0, 1)),
         # warp-specialised sweep on periodic axes (halo tiles: the producer's 16-byte copies)
         ((64, 18, 14), (1, 1, 1)), ((96, 20, 10), (0, 1, 0)), ((44, 24, 8), (1, 1, 0)), ((48, 12, 6), (1, 0, 1))]


def _close(got, ref, rtol=1e-5):
    scale = max(np.abs(ref).max(), 1e-30)
    err = np.abs(got - ref).max() / scale
    assert err <= rtol, f"max rel-to-max error {err:.3e}"


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("dims,periodic", CASES)
@pytest.mark.parametrize("omega", [1.0, 0.7])
def test_sweep_matches_oracle(O, dims, periodic, omega):
    from paper_2607_07687_gb300 import binding as G
    (bx, by, bz), b, p = random_fields(dims, periodic, seed=sum(dims) + int(omega * 10))
    out = t32(np.zeros_like(p))
    G.op_sweep(t32(bx), t32(by), t32(bz), t32(b), t32(p), out, omega, periodic)
    ref = O.sweep(p, b, bx, by, bz, omega, periodic)
    _close(host(out), ref)


@pytest.mark.parametrize("dims,periodic", CASES)
def test_sweep_single_launch_equals_two_launches(dims, periodic):
    """The single-launch sweep reproduces the colour-by-colour sweep bit for bit."""
    import torch
    from paper_2607_07687_gb300 import binding as G
    (bx, by, bz), b, p = random_fields(dims, periodic, seed=3 * sum(dims))
    args = [t32(a) for a in (bx, by, bz, b)]
    out = t32(np.zeros_like(p))
    G.op_sweep(*args, t32(p), out, 0.9, periodic)
    ref = t32(p)
    G.op_sweep_reference(*args, ref, 0.9, periodic)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


@pytest.mark.parametrize("zchunk", [1, 2, 3, 4, 5, 8, 13])
@pytest.mark.parametrize("dims,periodic", [((68, 18, 13), (0, 0, 0)), ((64, 20, 14), (1, 1, 1))])
def test_sweep_every_zchunk_equals_two_launches(dims, periodic, zchunk):
    """Every z-chunk depth of the pipelined sweep (chunks of one plane, odd and even
    plane counts, a ragged last chunk; each chunk restarts the plane ring with its
    two halo planes) reproduces the colour-by-colour sweep bit for bit."""
    import torch
    from paper_2607_07687_gb300 import binding as G
    nx, ny, nz = dims
    G.tune_import(f"z 0 {nx} {ny} {nz} {periodic[0]} {periodic[1]} {periodic[2]} {zchunk}\n")
    (bx, by, bz), b, p = random_fields(dims, periodic, seed=7 * sum(dims) + zchunk)
    args = [t32(a) for a in (bx, by, bz, b)]
    out = t32(np.zeros_like(p))
    G.op_sweep(*args, t32(p), out, 0.8, periodic)
    ref = t32(p)
    G.op_sweep_reference(*args, ref, 0.8, periodic)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


@pytest.mark.parametrize("dims,periodic,fac", [((70, 18, 14), (0, 0, 0), (2, 2, 2)),
                                               ((66, 18, 14), (1, 1, 1), (2, 1, 2)),
                                               ((34, 9, 12), (0, 0, 1), (2, 1, 2)),
                                               ((33, 20, 8), (0, 1, 0), (1, 2, 2)),
                                               ((40, 8, 6), (0, 0, 0), (2, 2, 1)),
                                               ((8, 6, 4), (0, 0, 0), (1, 1, 1)),
                                               ((64, 18, 14), (1, 1, 1), (2, 2, 2)),
                                               ((128, 40, 22), (0, 0, 0), (2, 2, 2)),
                                               ((96, 20, 30), (0, 1, 0), (2, 1, 2)),
                                               ((36, 12, 9), (0, 0, 0), (1, 2, 1)),
                                               ((260, 16, 12), (1, 0, 0), (1, 1, 2)),
                                               ((4, 4, 4), (1, 1, 1), (2, 2, 2))])
def test_residual_restrict_matches_oracle(O, dims, periodic, fac):
    from paper_2607_07687_gb300 import binding as G
    (bx, by, bz), b, p = random_fields(dims, periodic, seed=7 + sum(dims))
    nx, ny, nz = dims
    bc = t32(np.zeros((nz // fac[2], ny // fac[1], nx // fac[0])))
    rr = G.op_residual_restrict(t32(bx), t32(by), t32(bz), t32(b), t32(p), bc, fac, periodic,
                                want_norm=True)
    r = b - O.apply_A(p, bx, by, bz, periodic)
    _close(host(bc), O.restrict(r, fac))
    assert rr == pytest.approx(float(np.sum(r * r)), rel=1e-5)
    rn = G.op_residual_norm(t32(bx), t32(by), t32(bz), t32(b), t32(p), periodic)
    assert rn == pytest.approx(float(np.sum(r * r)), rel=1e-5)


@pytest.mark.parametrize("dims,fac", [((70, 18, 14), (2, 2, 2)), ((66, 18, 13), (2, 2, 1)),
                                      ((34, 9, 12), (1, 1, 2))])
def test_prolong_add_matches_oracle(O, dims, fac):
    from paper_2607_07687_gb300 import binding as G
    nx, ny, nz = dims
    rng = np.random.default_rng(1)
    p = f32(rng.standard_normal((nz, ny, nx)))
    e = f32(rng.standard_normal((nz // fac[2], ny // fac[1], nx // fac[0])))
    tp = t32(p)
    G.op_prolong_add(t32(e), tp, fac)
    _close(host(tp), O.prolong_add(p, e, fac), rtol=1e-6)


@pytest.mark.parametrize("dims,periodic,fac", [((70, 18, 14), (0, 0, 0), (2, 2, 2)),
                                               ((66, 18, 14), (1, 0, 1), (2, 1, 2)),
                                               ((34, 8, 12), (0, 1, 0), (1, 2, 1))])
def test_coarsen_coeffs_matches_oracle(O, dims, periodic, fac):
    from paper_2607_07687_gb300 import binding as G
    from paper_2607_07687_gb300 import inputs as I
    (bx, by, bz), _, _ = random_fields(dims, periodic, seed=11)
    nx, ny, nz = dims
    cshape = (nz // fac[2], ny // fac[1], nx // fac[0])
    out = [t32(np.zeros(cshape)) for _ in range(3)]
    G.op_coarsen_coeffs(t32(bx), t32(by), t32(bz), *out, fac, periodic)
    ref = O.coarsen_beta(*I.apply_walls(bx, by, bz, periodic), fac, periodic)
    for g, r in zip(out, ref):
        _close(host(g), r, rtol=1e-6)


def _face_sums(p, bx, by, bz, periodic):
    """Per cell: sum over its faces of beta_f |p_nb - p_I| and of beta_f (|p_nb| + |p_I|)
    (walls carry no face), the magnitudes the residual's roundings scale with."""
    diff = np.zeros_like(p)
    mag = np.zeros_like(p)
    for beta, ax, per in ((bx, 2, periodic[0]), (by, 1, periodic[1]), (bz, 0, periodic[2])):
        lo = beta.copy()
        hi = np.roll(beta, -1, axis=ax)
        if not per:
            idx = [slice(None)] * 3
            idx[ax] = 0
            lo[tuple(idx)] = 0.0
            idx[ax] = -1
            hi[tuple(idx)] = 0.0
        for face, nb in ((lo, np.roll(p, 1, axis=ax)), (hi, np.roll(p, -1, axis=ax))):
            diff += np.abs(face * (nb - p))
            mag += face * (np.abs(nb) + np.abs(p))
    return diff, mag


@pytest.mark.parametrize("dims,periodic", [((70, 18, 13), (0, 0, 0)), ((64, 16, 14), (1, 1, 1)),
                                           ((33, 20, 9), (0, 1, 0)), ((130, 40, 6), (1, 0, 0))])
def test_refinement_residual_definitions(O, dims, periodic):
    """r = b - A p of the FP64 refinement, on data where r is 1e-9 of b (the
    cancellation the refinement meets near convergence): the FP64 definition
    against the oracle's operator, within FP64 rounding of the face terms
    (2^-50 of sum beta (|p_nb| + |p_I|), since the oracle sums in another order);
    the solver's evaluation (FP64 differences, double-length FP32 products and
    sums) against the definition within 2^-40 of sum beta |p_nb - p_I| + |b|
    (about 2^-44 from the double-length arithmetic, 16x margin); cells with
    values beyond the FP32 exponent range fall back to the definition exactly."""
    import torch
    from paper_2607_07687_gb300 import binding as G
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    rng = np.random.default_rng(sum(dims))
    (bx, by, bz), _, _ = random_fields(dims, periodic, seed=sum(dims) + 1)
    z, y, x = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    p = 1e3 * np.sin(2 * np.pi * x / nx) * np.cos(2 * np.pi * y / ny) + 37.0 + rng.standard_normal(shape)
    p[1, 2, 3] = 3e39                                   # a difference beyond FP32 range: the FP64 path
    Ap = O.apply_A(p, bx, by, bz, periodic)
    b = Ap + 1e-9 * np.median(np.abs(Ap)) * rng.standard_normal(shape)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")
    tb, tp = T(b), T(p)
    beta = [t32(a) for a in (bx, by, bz)]
    r_def, r_df = torch.zeros_like(tb), torch.zeros_like(tb)
    r32 = torch.zeros(shape, dtype=torch.float32, device="cuda:0")
    rr_def = G.op_residual64(*beta, tb, tp, periodic, definition=1, r_out=r_def)
    rr_df = G.op_residual64(*beta, tb, tp, periodic, definition=0, r_out=r_df, r32_out=r32)
    r_def, r_df, r32 = host(r_def), host(r_df), host(r32)
    ref = b - Ap
    diff, mag = _face_sums(p, bx, by, bz, periodic)
    assert np.all(np.abs(r_def - ref) <= 2.0 ** -50 * (mag + np.abs(b)))
    assert np.all(np.abs(r_df - r_def) <= 2.0 ** -40 * (diff + np.abs(b)))
    far = (diff > 1e38)
    assert far.any() and np.array_equal(r_df[far], r_def[far])
    assert np.all(np.abs(r32 - r_df) <= 2.0 ** -24 * np.abs(r_df))     # r32: r rounded to FP32
    near = ~far
    print("max |r_df - r_def| / scale:", float(np.max(np.abs(r_df - r_def)[near] / (diff + np.abs(b))[near])),
          "r / b:", float(np.abs(ref[near]).max() / np.abs(b[near]).max()))
    assert rr_df == pytest.approx(float(np.sum(r32 * r32)), rel=1e-12)
    assert rr_def > 0
