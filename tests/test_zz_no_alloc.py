"""The residual-norm entry point that allocates nothing.

Real-time loops that must not meet the synchronisation of cudaMalloc /
cudaFree, and programs with a device-memory budget fixed up front, cannot let
a library allocate; gmg_op_residual_norm_noalloc serves them with a fixed
scratch array inside the library.  Checked here against gmg_op_residual_norm
(which allocates its scratch) on calls in a row with different inputs, and
for its size limit.  This file is collected last on purpose.

Tolerances.  Both entry points compute the same FP32 residuals (the operator's
roundings are spelled out identically in every kernel) and sum their squares
first in FP32, then in FP64.  On rows that are not a multiple of 4 cells both
run the same per-cell kernel, so the sums agree to FP64 rounding (rel 1e-12).
On rows of a multiple of 4 cells the allocating entry point runs the
z-marching kernel, which adds up to 16 squares in sequence per thread (an
FP32 partial off by at most 15 2^-24 relative), where the per-cell kernel
adds each warp's 32 squares as a five-level tree (at most 5 2^-24): the two
totals differ by at most 20 2^-24 < 1.2e-6 relative (checked at 2e-6)."""
import ctypes

import numpy as np
import pytest

from tests.gpu_common import random_fields, t32

pytestmark = pytest.mark.gpu


def _fields(dims, periodic, seed):
    (bx, by, bz), b, p = random_fields(dims, periodic, seed)
    return [t32(a) for a in (bx, by, bz, b, p)]


def test_matches_allocating_entry_point_twice():
    from paper_2607_07687_gb300 import binding as G
    cases = [((70, 19, 13), (0, 0, 0), 5, 1e-12), ((66, 18, 14), (1, 1, 1), 6, 1e-12),
             ((64, 16, 14), (1, 1, 1), 7, 2e-6), ((96, 24, 10), (0, 0, 0), 8, 2e-6)]
    for dims, periodic, seed, rel in cases:      # four calls in a row, different inputs
        f = _fields(dims, periodic, seed)
        ref = G.op_residual_norm(*f, periodic)
        got = G.op_residual_norm_noalloc(*f, periodic)
        assert ref > 0
        assert got == pytest.approx(ref, rel=rel, abs=0), (dims, got, ref)


def test_rejects_grids_beyond_the_static_scratch():
    from paper_2607_07687_gb300 import binding as G
    L = G.lib()
    rr = ctypes.c_double(-1.0)
    fake = ctypes.c_void_p(256)   # never dereferenced: the size check comes first
    rc = L.gmg_op_residual_norm_noalloc(1024, 256, 256, G._ivec((0, 0, 0)), fake, fake, fake, fake,
                                        fake, ctypes.byref(rr), None)
    assert rc == G.ERR_ARG
    assert "static scratch" in L.gmg_last_error(None).decode()
    assert rr.value == -1.0
