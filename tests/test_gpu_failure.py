"""Failure paths on the GPU, injected from the host (no GPU fault, trap or hang).

* A NaN written into the device-resident relaxation factor between two
  V-cycles (gmg_test_poison_omega): the control rule treats it as corrupt
  state, the solve returns GMG_ERR_DIVERGED with the iterate accepted before
  that cycle, and the handle's next solve is unaffected.
* The pipelined kernels' ring-slot waits cut to zero polls
  (gmg_test_ring_wait_tries): every such wait gives up at once, each block
  waits with its full limit for the copies it already issued and returns, and
  the solve reports GMG_ERR_CUDA ("timed out"); with the default limit back, a
  fresh handle solves normally and matches a solve made before the fault.
"""
import numpy as np
import pytest

from paper_2607_07687_gb300 import inputs as I
from tests.gpu_common import gpu_solve, host, t32

pytestmark = pytest.mark.gpu


def _channel():
    # rows of a multiple of 4 cells: the warp-specialised sweep and residual run
    return I.sphere_channel_problem(64, 32, 32, seed=1, radius=6.0, center_x=20.0)


def test_nan_omega_gives_diverged():
    import torch
    from paper_2607_07687_gb300 import binding as G
    prob = _channel()
    two, i2, _ = gpu_solve(prob, 1e-12, max_cycles=2, autotune=0)   # the iterate after two cycles
    assert i2.status == G.NOT_CONVERGED and i2.cycles == 2
    s = G.Solver(prob.dims, prob.periodic, autotune=0)
    try:
        s.set_coeffs(t32(prob.bx), t32(prob.by), t32(prob.bz))
        b = t32(prob.b)
        p = torch.zeros_like(b)
        s.test_poison_omega(3)
        info = s.solve(b, p, 1e-12)
        torch.cuda.synchronize()
        assert info.status == G.DIVERGED and info.cycles == 3, info.as_dict()
        hist, om, acc = s.history()
        assert list(acc) == [True, True, False]
        assert np.isnan(om[2])
        got = host(p)
        assert np.all(np.isfinite(got))
        assert np.array_equal(got, two)                 # the accepted iterate of cycle 2
        # one shot: the next solve of the same handle converges as usual
        p.zero_()
        again = s.solve(b, p, 1e-5)
        assert again.status == G.OK, again.as_dict()
    finally:
        s.close()


def test_ring_wait_timeout_is_reported():
    import torch
    from paper_2607_07687_gb300 import binding as G
    prob = _channel()
    before, ib, _ = gpu_solve(prob, 1e-5, autotune=0)
    assert ib.status == G.OK
    s = G.Solver(prob.dims, prob.periodic, autotune=0)
    try:
        s.set_coeffs(t32(prob.bx), t32(prob.by), t32(prob.bz))
        b = t32(prob.b)
        p = torch.zeros_like(b)
        G.test_ring_wait_tries(0)
        try:
            with pytest.raises(G.GmgError) as exc:
                s.solve(b, p, 1e-5)
        finally:
            G.test_ring_wait_tries(-1)
        assert "cuda error" in str(exc.value) and "timed out" in str(exc.value), str(exc.value)
    finally:
        s.close()
    torch.cuda.synchronize()                            # the context is still usable
    after, ia, _ = gpu_solve(prob, 1e-5, autotune=0)
    assert ia.status == G.OK and ia.cycles == ib.cycles
    assert np.array_equal(after, before)
