"""The residual-norm entry point that allocates nothing.

Callers recording CUDA graphs, real-time loops and programs with a fixed
device-memory budget cannot let a library call cudaMalloc;
gmg_op_residual_norm_noalloc serves them with a fixed scratch array inside the
library.  Checked here against gmg_op_residual_norm (which allocates its
scratch) on two calls in a row with different inputs, and for its size limit.
This file is collected last on purpose."""
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
    cases = [((70, 19, 13), (0, 0, 0), 5), ((66, 18, 14), (1, 1, 1), 6)]
    for dims, periodic, seed in cases:            # two calls in a row, different inputs
        f = _fields(dims, periodic, seed)
        ref = G.op_residual_norm(*f, periodic)
        got = G.op_residual_norm_noalloc(*f, periodic)
        assert ref > 0
        assert got == pytest.approx(ref, rel=1e-12, abs=0)


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
