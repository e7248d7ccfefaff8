"""C ABI checks that need no GPU: the library loads, exports every function
that include/gmg.h declares, and rejects bad arguments before touching CUDA."""
import ctypes

import pytest

from paper_2607_07687_gb300 import binding as G


@pytest.fixture(scope="module")
def L():
    from paper_2607_07687_gb300 import build
    build.build()
    return G.lib()


def test_exports_every_declared_function(L):
    names = G.declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    for core in ("gmg_create", "gmg_set_coeffs", "gmg_solve", "gmg_destroy", "gmg_batch_create",
                 "gmg_batch_set_coeffs", "gmg_batch_solve", "gmg_last_error"):
        assert core in names


def test_default_options(L):
    o = G.options()
    assert (o.nu1, o.nu2, o.nu_c, o.n_min, o.coarsen) == (2, 2, 16, 4, G.ANISO)
    assert (o.omega0, o.omega_min, o.shrink, o.grow) == (1.0, 0.25, 0.7, 1.1)


def _create(L, dims, periodic=(0, 0, 0), **kw):
    h = ctypes.c_void_p()
    coarsen = kw.pop("coarsen", "aniso")
    o = G.options(coarsen=coarsen, **kw)
    rc = L.gmg_create(ctypes.byref(h), *dims, G._ivec(periodic), ctypes.byref(o), None)
    return rc, L.gmg_last_error(None).decode()


@pytest.mark.parametrize("dims,periodic,kw,frag", [
    ((0, 8, 8), (0, 0, 0), {}, "dimension"),
    ((8, -1, 8), (0, 0, 0), {}, "dimension"),
    ((9, 8, 8), (1, 0, 0), {}, "periodic"),
    ((8, 8, 1), (0, 0, 1), {}, "periodic"),        # a 2D grid's length-1 axis cannot be periodic
    ((8, 8, 8), (0, 0, 0), {"nu2": 0}, "nu2"),
    ((8, 8, 8), (0, 0, 0), {"nu_c": 0}, "nu_c"),
    ((8, 8, 8), (0, 0, 0), {"max_cycles": 0}, "max_cycles"),
    ((8, 8, 8), (0, 0, 0), {"shrink": 1.5}, "shrink"),
    ((8, 8, 8), (0, 0, 0), {"n_min": 0}, "n_min"),
    ((8, 8, 8), (0, 0, 0), {"ir_inner_rtol": 0.0}, "ir_inner_rtol"),
    ((8, 8, 8), (0, 0, 0), {"coarse_mode": 2}, "coarse_mode"),
    ((8, 8, 8), (0, 0, 0), {"coarse_op": 2}, "coarse_op"),
    ((6, 6, 6), (0, 0, 0), {"coarse_mode": 1}, "two levels"),           # does not coarsen
    ((48, 48, 48), (0, 0, 0), {"coarse_mode": 1, "n_min": 16, "coarsen": "iso"}, "1024"),   # coarsest 24^3
])
def test_create_rejects(L, dims, periodic, kw, frag):
    rc, msg = _create(L, dims, periodic, **kw)
    assert rc == G.ERR_ARG
    assert frag in msg


def test_create_null_handle(L):
    o = G.options()
    assert L.gmg_create(None, 8, 8, 8, None, ctypes.byref(o), None) == G.ERR_ARG


def test_batch_create_rejects(L):
    b = ctypes.c_void_p()
    dims = G._ivec([8, 8, 8])
    o = G.options()
    assert L.gmg_batch_create(ctypes.byref(b), 0, dims, None, ctypes.byref(o), None) == G.ERR_ARG
    odd = G._ivec([7, 8, 8])                  # an odd periodic axis, checked before any allocation
    assert L.gmg_batch_create(ctypes.byref(b), 1, odd, G._ivec([1, 0, 0]), ctypes.byref(o), None) == G.ERR_ARG
    assert L.gmg_batch_last_error(None).decode()


def test_ops_reject_bad_arguments(L):
    fake = ctypes.c_void_p(16)   # never dereferenced: validation fails first
    per = G._ivec((0, 0, 0))
    # p_in aliasing p_out
    assert L.gmg_op_sweep(8, 8, 8, per, fake, fake, fake, fake, fake, fake, 1.0, None) == G.ERR_ARG
    # null input
    assert L.gmg_op_sweep(8, 8, 8, per, None, fake, fake, fake, fake, ctypes.c_void_p(32), 1.0,
                          None) == G.ERR_ARG
    # coarsening factor 3, or a factor that does not divide the axis
    assert L.gmg_op_prolong_add(8, 8, 8, G._ivec((3, 1, 1)), fake, fake, None) == G.ERR_ARG
    assert L.gmg_op_prolong_add(7, 8, 8, G._ivec((2, 1, 1)), fake, fake, None) == G.ERR_ARG
    assert L.gmg_op_coarsen_coeffs(8, 8, 8, per, G._ivec((2, 2, 4)), fake, fake, fake, fake, fake,
                                   fake, None) == G.ERR_ARG
    # residual norm without an output
    assert L.gmg_op_residual_norm(8, 8, 8, per, fake, fake, fake, fake, fake, None, None) == G.ERR_ARG
    assert L.gmg_op_residual_restrict(8, 8, 8, per, G._ivec((2, 2, 2)), fake, fake, fake, fake, fake,
                                      None, None, None) == G.ERR_ARG


def test_tune_table_round_trip(L):
    """The autotuner's table exports as text and imports back unchanged (no GPU involved)."""
    text = ("z 0 256 96 96 0 0 0 8\n"
            "z 2 128 48 48 0 0 0 12\n"
            "b 256 96 96 0 0 0 1 4 0 16 0 3 16\n"
            "c 64 123456789 457\n")
    G.tune_import(text)
    out = G.tune_export()
    for line in text.splitlines():
        assert line in out.splitlines()
    # a bottom line without the form field reads as the one-CTA form
    G.tune_import("b 128 96 96 0 0 0 1 4 0 16 0 4\n")
    assert "b 128 96 96 0 0 0 1 4 0 16 0 4 1" in G.tune_export().splitlines()
    # level 0 forgets the entry
    G.tune_import("b 128 96 96 0 0 0 1 4 0 16 0 0\n")
    assert not any(ln.startswith("b 128 96 96 ") for ln in G.tune_export().splitlines())
    # a replaced entry keeps one line per key
    G.tune_import("z 0 256 96 96 0 0 0 16\n")
    lines = G.tune_export().splitlines()
    assert "z 0 256 96 96 0 0 0 16" in lines and "z 0 256 96 96 0 0 0 8" not in lines
    # a batch's chunk policy: one line per (problem count, hash), replaced in place
    G.tune_import("c 64 123456789 0\n")
    lines = G.tune_export().splitlines()
    assert "c 64 123456789 0" in lines and "c 64 123456789 457" not in lines
    # too small a buffer is refused and reports the length
    n = ctypes.c_size_t(0)
    buf = ctypes.create_string_buffer(4)
    assert L.gmg_tune_export(buf, 4, ctypes.byref(n)) == G.ERR_ARG
    assert n.value == len(G.tune_export())


@pytest.mark.parametrize("bad", ["z 0 1 2\n", "q 1 2 3\n", "z 0 8 8 8 0 0 0 x\n", "b 1 2 3\n", "z 0 8 8 8 0 0 0 -4\n",
                                 "b 64 64 64 0 0 0 1 4 0 16 0 3 17\n", "b 64 64 64 0 0 0 1 4 0 16 0 3 0\n",
                                 "z 0 8 8 8 0 0 0 0\n", "c 1 5 2\n", "c 64 5\n", "c 64 5 -1\n"])
def test_tune_import_rejects_malformed(L, bad):
    before = G.tune_export()
    with pytest.raises(G.GmgError):
        G.tune_import("z 1 64 64 64 0 0 0 4\n" + bad)
    assert G.tune_export() == before              # nothing merged from a rejected table


def test_comparison_solvers_reject_bad_arguments(L):
    """The PCG and GMG-PCG entry points check their arguments before any CUDA work."""
    fake = ctypes.c_void_p(16)
    info = G.Info()
    assert L.gmg_pcg_solve(None, fake, fake, 1e-6, 10, ctypes.byref(info)) == G.ERR_ARG
    assert L.gmg_gmgpcg_solve(None, fake, fake, 1e-6, ctypes.byref(info)) == G.ERR_ARG
    h = ctypes.c_void_p(8)   # never dereferenced: a non-positive tolerance is refused first
    assert L.gmg_pcg_solve(h, fake, fake, 0.0, 10, ctypes.byref(info)) == G.ERR_ARG
    assert L.gmg_gmgpcg_solve(h, fake, fake, -1.0, ctypes.byref(info)) == G.ERR_ARG
    assert L.gmg_pcg_solve(h, None, fake, 1e-6, 10, ctypes.byref(info)) == G.ERR_ARG
