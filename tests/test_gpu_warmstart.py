"""Parity of the warm-start network's kernels (BF16 tensor-core convolutions,
FP32 sums) with the FP64 network oracle, and the gain of the trained net.

Inputs are rounded to BF16 on the host before both sides see them, so the
oracle computes exactly on the values the kernels multiply.  Tolerances:
one BF16 rounding of each output (relative 2^-9, checked as 2^-8) for a
single kernel; FP32 accumulation error (~1e-4 of the sum of |terms|) for the
weight gradient; for the whole network a relative L2 error of the output
within half the chain of BF16 roundings along the longest path, and for
each parameter gradient that chain's error amplified by the measured
cancellation ratio of its sum over cells (derived in
test_network_forward_and_gradients_match_oracle).
"""
import numpy as np
import pytest

from oracle import warmstart_oracle as O

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8


def _torch():
    import torch
    return torch


def bf(a):
    """Host float64 values of the BF16 rounding of a."""
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def to_cl(a, cs=None, off=0):
    """[C][D][H][W] host array -> channels-last BF16 device tensor with cs channels."""
    torch = _torch()
    c = a.shape[0]
    cs = cs or c
    out = np.zeros((int(np.prod(a.shape[1:])), cs), dtype=np.float32)
    out[:, off:off + c] = a.reshape(c, -1).T
    return torch.from_numpy(out).to("cuda:0").to(torch.bfloat16)


def from_cl(t, shape, c0=0, c=None):
    """Channels-last device tensor -> [C][D][H][W] float64 host array."""
    a = t.float().cpu().numpy().astype(np.float64)
    c = c or a.shape[1] - c0
    return np.ascontiguousarray(a[:, c0:c0 + c].T.reshape((c,) + tuple(shape)))


def ptr(t, off=0):
    import ctypes
    return ctypes.c_void_p(t.data_ptr() + off * t.element_size())


def stream():
    import ctypes
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def call(name, *args):
    from paper_2607_07687_gb300 import binding as G
    G.net_call(name, *args)


def pack_weights(w):
    """[co][ci][3][3][3] -> FP32 device tensor packed [27][co][ci], its BF16 copy and flipped copy."""
    torch = _torch()
    co, ci = w.shape[:2]
    wp = np.ascontiguousarray(w.reshape(co, ci, 27).transpose(2, 0, 1), dtype=np.float32)
    w32 = torch.from_numpy(wp.ravel()).to("cuda:0")
    z = torch.zeros_like(w32)
    m, v = torch.zeros_like(w32), torch.zeros_like(w32)
    wb = torch.zeros((27, co, ci), dtype=torch.bfloat16, device="cuda:0")
    wt = torch.zeros((27, ci, co), dtype=torch.bfloat16, device="cuda:0")
    call("gmg_net_adam", w32.numel(), ptr(w32), ptr(z), ptr(m), ptr(v), 1, 0.0, 0.9, 0.999, 1e-8, ptr(wb), ptr(wt),
         co, ci, stream())
    return w32, wb, wt


def rand_w(rng, co, ci):
    return bf(rng.standard_normal((co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci)))


# ------------------------------------------------------------------ convolution

@pytest.mark.parametrize("ci,co", [(16, 16), (16, 32), (32, 48), (32, 64), (96, 32), (48, 96), (64, 16)])
def test_conv3_forward(ci, co):
    torch = _torch()
    rng = np.random.default_rng(ci * 100 + co)
    shape = (3, 6, 40)                         # ragged against the 4 x 32 tile
    x = bf(rng.standard_normal((ci,) + shape))
    w = rand_w(rng, co, ci)
    b = rng.standard_normal(co).astype(np.float32).astype(np.float64)
    _, wb, _ = pack_weights(w)
    bias = torch.from_numpy(b.astype(np.float32)).to("cuda:0")
    xt = to_cl(x)
    for relu in (0, 1):
        y = torch.zeros((xt.shape[0], co), dtype=torch.bfloat16, device="cuda:0")
        call("gmg_net_conv3", shape[0], shape[1], shape[2], ptr(xt), ci, ci, ptr(wb), ptr(bias), co, relu, ptr(y),
             co, 0, stream())
        ref = O.conv3(x, w, b)
        if relu:
            ref = O.relu(ref)
        got = from_cl(y, shape)
        err = np.abs(got - ref)
        assert np.all(err <= U_BF16 * np.abs(ref) + 1e-5 * np.abs(ref).max()), (relu, err.max())


@pytest.mark.parametrize("co", [16, 32, 64])
@pytest.mark.parametrize("shape", [(9, 6, 40), (13, 5, 150)])
def test_conv3_forward_z_marching(co, shape):
    """Layers with 16 input channels march a column of planes per block (a ring of
    input planes, double-buffered accumulators): grids of 9 and 13 planes split
    into several z-chunks with a ragged last one, rows of 40 and of 150 cells (a
    full tile and a tail), every output against the FP64 oracle."""
    torch = _torch()
    ci = 16
    rng = np.random.default_rng(co * 10 + shape[0])
    x = bf(rng.standard_normal((ci,) + shape))
    w = rand_w(rng, co, ci)
    b = rng.standard_normal(co).astype(np.float32).astype(np.float64)
    _, wb, _ = pack_weights(w)
    bias = torch.from_numpy(b.astype(np.float32)).to("cuda:0")
    xt = to_cl(x)
    y = torch.zeros((xt.shape[0], co), dtype=torch.bfloat16, device="cuda:0")
    call("gmg_net_conv3", shape[0], shape[1], shape[2], ptr(xt), ci, ci, ptr(wb), ptr(bias), co, 1, ptr(y),
         co, 0, stream())
    ref = O.relu(O.conv3(x, w, b))
    got = from_cl(y, shape)
    err = np.abs(got - ref)
    assert np.all(err <= U_BF16 * np.abs(ref) + 1e-5 * np.abs(ref).max()), err.max()


@pytest.mark.parametrize("ci,co", [(16, 16), (48, 16)])
def test_conv3_full_size_sampled(ci, co):
    """The network's level-0 layers at their full size (192 x 64 x 64: the 16 -> 16
    layer in the z-marching form with its ragged last z-chunk, the decoder's
    48 -> 16 in the one-plane form): 4096 sampled outputs against the
    convolution's definition evaluated in FP64 at those cells (zero padding)."""
    torch = _torch()
    rng = np.random.default_rng(ci * 7 + co)
    shape = (64, 64, 192)
    x = bf(rng.standard_normal((ci,) + shape))
    w = rand_w(rng, co, ci)
    b = rng.standard_normal(co).astype(np.float32).astype(np.float64)
    _, wb, _ = pack_weights(w)
    bias = torch.from_numpy(b.astype(np.float32)).to("cuda:0")
    xt = to_cl(x)
    y = torch.zeros((xt.shape[0], co), dtype=torch.bfloat16, device="cuda:0")
    call("gmg_net_conv3", shape[0], shape[1], shape[2], ptr(xt), ci, ci, ptr(wb), ptr(bias), co, 0, ptr(y),
         co, 0, stream())
    got = y.float().cpu().numpy().astype(np.float64).reshape(shape + (co,))
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    zs, ys, xs = (rng.integers(0, n, 4096) for n in shape)
    ref = np.stack([np.einsum("ocijk,cijk->o", w, xp[:, z:z + 3, yy:yy + 3, xx:xx + 3]) + b
                    for z, yy, xx in zip(zs, ys, xs)])
    err = np.abs(got[zs, ys, xs] - ref)
    assert np.all(err <= U_BF16 * np.abs(ref) + 1e-5 * np.abs(ref).max()), err.max()


@pytest.mark.parametrize("shape", [(2, 5, 192), (2, 5, 300)])
@pytest.mark.parametrize("ci,co", [(16, 16), (32, 64), (96, 32), (48, 96)])
def test_conv3_forward_long_rows(ci, co, shape):
    """Rows longer than one 128-cell tile: x = 192 (a full tile and a 64-cell tail)
    and x = 300 (two full tiles and a 44-cell tail), five rows (a ragged group of
    the four row tiles a CTA takes).  Every output, including the two on each side
    of a tile boundary whose window reaches into the neighbouring tile, against
    the FP64 oracle."""
    torch = _torch()
    rng = np.random.default_rng(ci * 1000 + co + shape[2])
    x = bf(rng.standard_normal((ci,) + shape))
    w = rand_w(rng, co, ci)
    b = rng.standard_normal(co).astype(np.float32).astype(np.float64)
    _, wb, _ = pack_weights(w)
    bias = torch.from_numpy(b.astype(np.float32)).to("cuda:0")
    xt = to_cl(x)
    y = torch.zeros((xt.shape[0], co), dtype=torch.bfloat16, device="cuda:0")
    call("gmg_net_conv3", shape[0], shape[1], shape[2], ptr(xt), ci, ci, ptr(wb), ptr(bias), co, 1, ptr(y),
         co, 0, stream())
    ref = O.relu(O.conv3(x, w, b))
    got = from_cl(y, shape)
    err = np.abs(got - ref)
    assert np.all(err <= U_BF16 * np.abs(ref) + 1e-5 * np.abs(ref).max()), err.max()
    edges = [127, 128, 255, 256] if shape[2] > 256 else [127, 128]
    assert np.allclose(got[..., edges], ref[..., edges], rtol=U_BF16, atol=1e-5 * np.abs(ref).max())


def test_conv3_channel_offsets_and_bias_free():
    """Input read from channels 16..47 of a 48-channel buffer, output written to
    channels 16..79 of an 80-channel buffer; the other channels stay untouched."""
    torch = _torch()
    rng = np.random.default_rng(7)
    shape = (4, 5, 33)
    ci, co = 32, 64
    x = bf(rng.standard_normal((ci,) + shape))
    junk = bf(rng.standard_normal((16,) + shape))
    w = rand_w(rng, co, ci)
    _, wb, _ = pack_weights(w)
    xt = to_cl(x, 48, 16)
    xt[:, :16] = to_cl(junk)
    y = torch.full((xt.shape[0], 80), 3.0, dtype=torch.bfloat16, device="cuda:0")
    call("gmg_net_conv3", *shape, ptr(xt, 16), 48, ci, ptr(wb), None, co, 0, ptr(y), 80, 16, stream())
    ref = O.conv3(x, w, np.zeros(co))
    got = from_cl(y, shape, 16, co)
    assert np.all(np.abs(got - ref) <= U_BF16 * np.abs(ref) + 1e-5 * np.abs(ref).max())
    yh = y.float().cpu().numpy()
    assert np.all(yh[:, :16] == 3.0)


@pytest.mark.parametrize("ci,co", [(16, 16), (32, 64), (96, 32), (48, 16)])
def test_conv3_input_gradient(ci, co):
    """The forward kernel on the flipped transposed weights is the adjoint."""
    torch = _torch()
    rng = np.random.default_rng(ci + 7 * co)
    shape = (5, 7, 36)
    w = rand_w(rng, co, ci)
    g = bf(rng.standard_normal((co,) + shape))
    _, _, wt = pack_weights(w)
    gt = to_cl(g)
    gx = torch.zeros((gt.shape[0], ci), dtype=torch.bfloat16, device="cuda:0")
    call("gmg_net_conv3", *shape, ptr(gt), co, co, ptr(wt), None, ci, 0, ptr(gx), ci, 0, stream())
    ref = O.conv3_backward(np.zeros((ci,) + shape), w, g)[0]
    got = from_cl(gx, shape)
    assert np.all(np.abs(got - ref) <= U_BF16 * np.abs(ref) + 1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("shape", [(2, 5, 192), (2, 5, 300)])
@pytest.mark.parametrize("ci,co", [(16, 16), (32, 64), (48, 16)])
def test_conv3_input_gradient_long_rows(ci, co, shape):
    """The adjoint convolution on rows longer than one 128-cell tile (x = 192 and a
    ragged x = 300)."""
    torch = _torch()
    rng = np.random.default_rng(ci + 7 * co + shape[2])
    w = rand_w(rng, co, ci)
    g = bf(rng.standard_normal((co,) + shape))
    _, _, wt = pack_weights(w)
    gt = to_cl(g)
    gx = torch.zeros((gt.shape[0], ci), dtype=torch.bfloat16, device="cuda:0")
    call("gmg_net_conv3", *shape, ptr(gt), co, co, ptr(wt), None, ci, 0, ptr(gx), ci, 0, stream())
    ref = O.conv3_backward(np.zeros((ci,) + shape), w, g)[0]
    got = from_cl(gx, shape)
    assert np.all(np.abs(got - ref) <= U_BF16 * np.abs(ref) + 1e-5 * np.abs(ref).max())


@pytest.mark.parametrize("ci,co,shape", [(16, 16, (3, 6, 40)), (48, 32, (4, 8, 12)), (96, 64, (2, 4, 20)),
                                         (32, 32, (16, 16, 16)), (16, 16, (2, 5, 300)), (32, 64, (2, 3, 192))])
def test_conv3_weight_gradient(ci, co, shape):
    torch = _torch()
    rng = np.random.default_rng(ci * 3 + co)
    x = bf(rng.standard_normal((ci,) + shape))
    g = bf(rng.standard_normal((co,) + shape))
    xt, gt = to_cl(x), to_cl(g)
    dw = torch.full((27 * co * ci,), 0.5, dtype=torch.float32, device="cuda:0")   # accumulates
    db = torch.full((co,), 0.25, dtype=torch.float32, device="cuda:0")
    call("gmg_net_conv3_wgrad", *shape, ptr(xt), ci, ci, ptr(gt), co, co, ptr(dw), ptr(db), stream())
    _, gw, gb = O.conv3_backward(x, np.zeros((co, ci, 3, 3, 3)), g)
    _, aw, ab = O.conv3_backward(np.abs(x), np.zeros((co, ci, 3, 3, 3)), np.abs(g))
    got = dw.cpu().numpy().astype(np.float64).reshape(27, co, ci).transpose(1, 2, 0).reshape(co, ci, 3, 3, 3)
    assert np.all(np.abs(got - 0.5 - gw) <= 1e-4 * aw + 1e-6)
    assert np.all(np.abs(db.cpu().numpy() - 0.25 - gb) <= 1e-4 * ab + 1e-6)


# ------------------------------------------------------------------ elementwise

def test_pool_upsample_relu_kernels():
    torch = _torch()
    rng = np.random.default_rng(11)
    C, shape = 16, (6, 10, 14)
    cshape = tuple(s // 2 for s in shape)
    x = bf(rng.standard_normal((C,) + shape))
    xt = to_cl(x, 32, 16)
    # pool into channels 8..23 of a 32-channel coarse buffer
    y = torch.zeros((int(np.prod(cshape)), 32), dtype=torch.bfloat16, device="cuda:0")
    call("gmg_net_pool2", *shape, ptr(xt, 16), 32, C, ptr(y), 32, 8, stream())
    ref = O.pool2(x)
    assert np.all(np.abs(from_cl(y, cshape, 8, C) - ref) <= U_BF16 * np.abs(ref) + 1e-7)
    # up2 (a copy: exact)
    xc = bf(rng.standard_normal((C,) + cshape))
    xct = to_cl(xc)
    yu = torch.zeros((int(np.prod(shape)), 48), dtype=torch.bfloat16, device="cuda:0")
    call("gmg_net_up2", *cshape, ptr(xct), C, C, ptr(yu), 48, 32, stream())
    assert np.array_equal(from_cl(yu, shape, 32, C), O.up2(xc))
    # up2 backward from channels 16..31 of a 48-channel gradient
    gy = bf(rng.standard_normal((C,) + shape))
    gyt = to_cl(gy, 48, 16)
    gx = torch.zeros((int(np.prod(cshape)), C), dtype=torch.bfloat16, device="cuda:0")
    call("gmg_net_up2_backward", *cshape, ptr(gyt), 48, 16, C, ptr(gx), C, stream())
    ref = O.up2_backward(gy)
    assert np.all(np.abs(from_cl(gx, cshape) - ref) <= U_BF16 * np.abs(ref) + 1e-6)
    # pool backward plus a skip gradient taken from channels 32..47
    gc = bf(rng.standard_normal((C,) + cshape))
    add = bf(rng.standard_normal((C,) + shape))
    gct, addt = to_cl(gc), to_cl(add, 48, 32)
    gf = torch.zeros((int(np.prod(shape)), C), dtype=torch.bfloat16, device="cuda:0")
    call("gmg_net_pool2_backward", *shape, ptr(gct), C, C, ptr(gf), C, ptr(addt), 48, 32, stream())
    ref = O.pool2_backward(gc) + add
    assert np.all(np.abs(from_cl(gf, shape) - ref) <= U_BF16 * np.abs(ref) + 1e-7)
    # relu backward against an activation read from channels 16..31
    act = O.relu(bf(rng.standard_normal((C,) + shape)))
    actt = to_cl(act, 32, 16)
    g = bf(rng.standard_normal((C,) + shape))
    gt = to_cl(g)
    call("gmg_net_relu_backward", *shape, ptr(gt), C, ptr(actt, 16), 32, C, stream())
    assert np.array_equal(from_cl(gt, shape), g * (act > 0))


def beta_mean(bx, by, bz, periodic):
    """Mean of each cell's six face coefficients; faces on walls are zero."""
    out = np.zeros(bx.shape)
    for axis_arr, ax, per in ((bx, 2, periodic[0]), (by, 1, periodic[1]), (bz, 0, periodic[2])):
        lo = axis_arr.copy()
        hi = np.roll(axis_arr, -1, axis=ax)
        if not per:
            idx = [slice(None)] * 3
            idx[ax] = 0
            lo[tuple(idx)] = 0.0
            idx[ax] = -1
            hi[tuple(idx)] = 0.0
        out += lo + hi
    return out / 6.0


@pytest.mark.parametrize("periodic", [(False, False, False), (True, False, True)])
@pytest.mark.parametrize("with_prev", [True, False])
def test_pack_input(periodic, with_prev, oracle):
    """Input channels against the oracle's features, with the residual
    r = b - A p_prev from the FP64 solver oracle's operator."""
    import ctypes
    torch = _torch()
    rng = np.random.default_rng(5)
    shape = (4, 6, 8)
    b = rng.standard_normal(shape).astype(np.float32)
    pp = rng.standard_normal(shape).astype(np.float32) if with_prev else np.zeros(shape, np.float32)
    bx, by, bz = (rng.uniform(0, 1, shape).astype(np.float32) for _ in range(3))
    T = lambda a: torch.from_numpy(a).to("cuda:0")
    x0 = torch.full((b.size, 16), 9.0, dtype=torch.bfloat16, device="cuda:0")
    s = torch.zeros(2, dtype=torch.float32, device="cuda:0")
    red = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    per = (ctypes.c_int * 3)(*[int(v) for v in periodic])
    bt, pt, bxt, byt, bzt = T(b), T(pp), T(bx), T(by), T(bz)
    call("gmg_net_pack_input", *shape, ptr(bt), ptr(pt) if with_prev else None, ptr(bxt), ptr(byt), ptr(bzt), per,
         ptr(x0), ptr(s), ptr(red), stream())
    f64 = [a.astype(np.float64) for a in (b, pp, bx, by, bz)]
    bm = beta_mean(*f64[2:], periodic)
    r = f64[0] - oracle.apply_A(f64[1], *f64[2:], periodic=periodic)
    ref, sref = O.features(f64[0], bm, f64[1], r)
    sh = s.cpu().numpy()
    assert float(sh[0]) == pytest.approx(sref, rel=1e-6)
    assert float(sh[1]) == pytest.approx(float(np.sqrt(np.mean(r * r))), rel=1e-5)
    got = from_cl(x0, shape)
    assert np.all(np.abs(got[:4] - ref) <= U_BF16 * np.abs(ref) + 1e-5)
    assert np.all(got[4:] == 0.0)


def test_head_loss_and_head_backward():
    torch = _torch()
    rng = np.random.default_rng(9)
    shape = (4, 8, 8)
    n = int(np.prod(shape))
    h = O.relu(bf(rng.standard_normal((16,) + shape)))
    w = rng.standard_normal(16).astype(np.float32)
    bb = np.array([0.3], dtype=np.float32)
    ht = to_cl(h)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda:0")
    wt, bt = T(w), T(bb)
    out = torch.zeros(n, dtype=torch.float32, device="cuda:0")
    call("gmg_net_head", *shape, ptr(ht), 16, ptr(wt), ptr(bt), ptr(out), stream())
    ref = np.einsum("i,izyx->zyx", w.astype(np.float64), h) + 0.3
    got = out.cpu().numpy().astype(np.float64).reshape(shape)
    np.testing.assert_allclose(got, ref, rtol=1e-5, atol=1e-5)
    # loss of out + p_prev / s against target / s, with and without p_prev
    target = rng.standard_normal(shape).astype(np.float32)
    pprev = rng.standard_normal(shape).astype(np.float32)
    s = np.float32(2.5)
    gout = torch.zeros_like(out)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    red = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    tt, st, pt = T(target), T(np.array([s])), T(pprev)
    for prev in (None, pt):
        call("gmg_net_loss", *shape, ptr(out), ptr(tt), ptr(prev) if prev is not None else None, ptr(st), ptr(gout),
             ptr(loss), ptr(red), stream())
        p0 = float(s) * got + (pprev.astype(np.float64) if prev is not None else 0.0)
        lref, gref = O.loss_and_grad_out(p0, target.astype(np.float64))
        assert float(loss.item()) == pytest.approx(lref, rel=1e-5)
        # d loss / d out = s * d loss / d p0
        np.testing.assert_allclose(gout.cpu().numpy().reshape(shape), float(s) * gref, rtol=1e-4,
                                   atol=1e-6 * np.abs(gref).max() * float(s))
    # unscale: p0 = s * out + p_prev
    p0t = torch.zeros_like(out)
    call("gmg_net_unscale", n, ptr(out), ptr(st), ptr(pt), ptr(p0t), stream())
    np.testing.assert_allclose(p0t.cpu().numpy().reshape(shape), float(s) * got + pprev, rtol=1e-6, atol=1e-6)
    # head backward
    go = rng.standard_normal(shape).astype(np.float32)
    gh = torch.zeros((n, 16), dtype=torch.bfloat16, device="cuda:0")
    dw = torch.zeros(16, dtype=torch.float32, device="cuda:0")
    db = torch.zeros(1, dtype=torch.float32, device="cuda:0")
    got_ = T(go)
    call("gmg_net_head_backward", *shape, ptr(got_), ptr(ht), 16, ptr(wt), ptr(gh), ptr(dw), ptr(db), stream())
    g64 = go.astype(np.float64)
    refgh = w.astype(np.float64)[:, None, None, None] * g64[None]
    assert np.all(np.abs(from_cl(gh, shape) - refgh) <= U_BF16 * np.abs(refgh) + 1e-7)
    aw = np.einsum("zyx,izyx->i", np.abs(g64), np.abs(h))
    assert np.all(np.abs(dw.cpu().numpy() - np.einsum("zyx,izyx->i", g64, h)) <= 1e-5 * aw + 1e-6)
    assert float(db.item()) == pytest.approx(g64.sum(), abs=1e-5 * np.abs(g64).sum())


@pytest.mark.parametrize("periodic", [(False, False, False), (True, True, False)])
def test_residual_loss_kernel(periodic, oracle):
    """Loss and gradient of the residual loss against the oracle (FP64 operator)
    on the same FP32 inputs; r is O(b) here, so FP32 keeps ~1e-6 relative."""
    import ctypes
    torch = _torch()
    rng = np.random.default_rng(13)
    shape = (4, 6, 8)
    n = int(np.prod(shape))
    f = lambda a: a.astype(np.float32)
    b, out, pp = f(rng.standard_normal(shape)), f(rng.standard_normal(shape)), f(rng.standard_normal(shape))
    bx, by, bz = (f(rng.uniform(0.1, 1.0, shape)) for _ in range(3))
    sc = np.float32(0.7)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda:0")
    ts = [T(a) for a in (b, out, pp, bx, by, bz, np.array([sc]))]
    work = torch.zeros(2 * n, dtype=torch.float32, device="cuda:0")
    gout = torch.zeros(n, dtype=torch.float32, device="cuda:0")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda:0")
    red = torch.zeros(2, dtype=torch.float64, device="cuda:0")
    per = (ctypes.c_int * 3)(*[int(v) for v in periodic])
    call("gmg_net_residual_loss", *shape, ptr(ts[1]), ptr(ts[2]), ptr(ts[6]), ptr(ts[0]), ptr(ts[3]), ptr(ts[4]),
         ptr(ts[5]), per, ptr(work), ptr(gout), ptr(loss), ptr(red), stream())
    f64 = [a.astype(np.float64) for a in (b, out, pp, bx, by, bz)]
    A = lambda v: oracle.apply_A(v, *f64[3:], periodic=periodic)
    p0 = f64[2] + float(sc) * f64[1]
    lref, gref = O.residual_loss_and_grad(p0, f64[0], A)
    assert float(loss.item()) == pytest.approx(lref, rel=1e-5)
    g = gout.cpu().numpy().astype(np.float64).reshape(shape)
    np.testing.assert_allclose(g, float(sc) * gref, rtol=1e-4, atol=1e-5 * np.abs(gref).max())


def test_adam_matches_oracle_and_packs():
    torch = _torch()
    rng = np.random.default_rng(12)
    co, ci = 16, 32
    w0 = rng.standard_normal((27, co, ci)).astype(np.float32)
    w = torch.from_numpy(w0.ravel().copy()).to("cuda:0")
    m, v = torch.zeros_like(w), torch.zeros_like(w)
    wb = torch.zeros((27, co, ci), dtype=torch.bfloat16, device="cuda:0")
    wt = torch.zeros((27, ci, co), dtype=torch.bfloat16, device="cuda:0")
    params = {"a": w0.ravel().astype(np.float64)}
    state = {}
    for t in range(1, 4):
        g = rng.standard_normal(w0.size).astype(np.float32)
        gt = torch.from_numpy(g).to("cuda:0")
        call("gmg_net_adam", w.numel(), ptr(w), ptr(gt), ptr(m), ptr(v), t, 1e-2, 0.9, 0.999, 1e-8, ptr(wb), ptr(wt),
             co, ci, stream())
        O.adam_step(params, {"a": g.astype(np.float64)}, state, lr=1e-2)
    got = w.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(got, params["a"], rtol=0, atol=1e-5)
    wf = got.astype(np.float32).reshape(27, co, ci)
    assert np.array_equal(wb.float().cpu().numpy(), bf(wf).astype(np.float32))
    flip = np.ascontiguousarray(wf[::-1].transpose(0, 2, 1))
    assert np.array_equal(wt.float().cpu().numpy(), bf(flip).astype(np.float32))


# ------------------------------------------------------------------ whole network

def _net_and_inputs(seed=21, dims=(32, 16, 16)):
    torch = _torch()
    from paper_2607_07687_gb300.warmstart import WarmStartNet
    rng = np.random.default_rng(seed)
    nx, ny, nz = dims
    shape = (nz, ny, nx)
    params = O.init_params(seed)
    for k in params:
        if k.endswith(".b"):
            params[k] = rng.standard_normal(params[k].shape) * 0.05
    net = WarmStartNet(dims, seed=0)
    net.set_weights(params)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda:0")
    b = rng.standard_normal(shape)
    pp = rng.standard_normal(shape)
    coef = [rng.uniform(0.2, 1.0, shape) for _ in range(3)]
    target = rng.standard_normal(shape) + 0.5 * pp
    dev = [T(a) for a in (b, *coef, pp, target)]
    # the kernels compute with BF16 weights, FP32 biases and head
    used = {}
    for k, v in params.items():
        used[k] = bf(v) if (k.endswith(".w") and not k.startswith("out")) else v.astype(np.float32).astype(np.float64)
    return net, dev, used, shape


# BF16 roundings on the longest path into a weight gradient: eleven forward stages
# (packed input, ten convolutions and poolings/upsamplings folded in) and eleven
# backward stages (head backward, ten input gradients), each rounding to BF16
U_ROUND = 2.0 ** -9
CHAIN = 22

LAYER_INPUT = {"e0a": "x0", "e0b": "e0a", "e1a": "p1", "e1b": "e1a", "e2a": "p2", "e2b": "e2a", "d1a": "c1",
               "d1b": "d1a", "d0a": "c0", "d0b": "d0a"}


@pytest.mark.parametrize("dims", [(32, 16, 16), (192, 16, 16)])
def test_network_forward_and_gradients_match_oracle(dims):
    """The whole network (forward, loss gradient, backward) against the FP64 oracle,
    at 32x16x16 and at 192x16x16 (level-0 rows of 192 cells: a full 128-cell tile
    and a tail).  Bound of each parameter gradient, derived, not fitted: every
    gradient sums products x g over cells, where x (the layer's input) and g (its
    output gradient) each come through a chain of BF16 roundings; with CHAIN
    roundings of relative size U_ROUND along the longest path the products are off
    by at most CHAIN * U_ROUND relative, and the sum by that times the layer's
    cancellation ratio kappa = |sum |x| |g|| / |sum x g| (L2 over the gradient's
    entries, from the oracle's own activations and gradients)."""
    net, (b, bx, by, bz, pp, target), used, shape = _net_and_inputs(dims=dims)
    net.pack(b, bx, by, bz, pp)
    net.forward()
    x0 = from_cl(net.a["x0"], shape)[:4]
    out_ref, cache = O.forward(used, x0)
    out = net.out.cpu().numpy().astype(np.float64).reshape(shape)
    fwd = np.linalg.norm(out - out_ref) / np.linalg.norm(out_ref)
    assert fwd <= CHAIN / 2 * U_ROUND, fwd
    net.loss(target, pp)
    s = float(net.s[0].item())
    # the oracle's loss gradient at the oracle's own prediction, in units of s
    pq = pp.cpu().numpy().astype(np.float64).reshape(shape) / s
    _, gref = O.loss_and_grad_out(out_ref + pq, target.cpu().numpy().astype(np.float64).reshape(shape) / s)
    net.backward()
    grads = net.gradients()
    rec = {}
    ref = O.backward(used, cache, gref, record=rec)
    # the loss ignores a constant shift of out, so d loss / d out.b = sum(gout) is 0
    assert abs(grads["out.b"][0]) <= 1e-5 * np.abs(gref).sum()
    kappa = {}
    for name, inp in LAYER_INPUT.items():
        x, g = cache[inp], rec[name]
        _, aw, ab = O.conv3_backward(np.abs(x), np.zeros_like(ref[name + ".w"]), np.abs(g))
        kappa[name + ".w"] = np.linalg.norm(aw) / np.linalg.norm(ref[name + ".w"])
        kappa[name + ".b"] = np.linalg.norm(ab) / max(np.linalg.norm(ref[name + ".b"]), 1e-300)
    h = cache["d0b"]
    kappa["out.w"] = (np.linalg.norm(np.einsum("zyx,izyx->i", np.abs(gref), np.abs(h)))
                      / np.linalg.norm(ref["out.w"]))
    report, bad = {}, {}
    for k in ref:
        if k == "out.b":
            continue
        a, r = grads[k].ravel(), ref[k].ravel()
        rel = np.linalg.norm(a - r) / max(np.linalg.norm(r), 1e-30)
        bound = CHAIN * U_ROUND * kappa[k]
        report[k] = (round(rel, 5), round(bound, 5), round(kappa[k], 2))
        if not rel <= bound:
            bad[k] = report[k]
    print("dims", dims, "forward rel L2", fwd, "(bound", CHAIN / 2 * U_ROUND, ")")
    print("gradient rel L2 / bound / kappa:", report)
    assert not bad, bad


def test_training_lowers_the_loss():
    """Adam steps on one (input, target) pair drive the loss down."""
    net, (b, bx, by, bz, pp, target), _, _ = _net_and_inputs(seed=22)
    losses = [net.train_step(b, bx, by, bz, pp, target) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])


def test_warm_start_gain_on_vortex_sequence():
    """A net trained on GMG solves of one vortex sequence (seed 31) gives a
    held-out sequence (seed 4) initial guesses that save V-cycles against the
    zero guess, at the same tolerance."""
    torch = _torch()
    from paper_2607_07687_gb300 import binding as G
    from paper_2607_07687_gb300 import inputs as I
    from paper_2607_07687_gb300.warmstart import WarmStartNet
    geo = dict(nx=64, ny=32, nz=32, radius=4.0, center_x=16.0, blob_sigma=3.0)
    tol = 1e-5
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to("cuda:0")

    def frames(seed, count):
        seq = I.VortexSequence(seed=seed, **geo)
        out = []
        for _ in range(count):
            out.append(seq.problem())
            seq.advance()
        return out

    train = frames(31, 24)
    held = frames(4, 8)
    dims = train[0].dims
    solver = G.Solver(dims, (False, False, False), precision="fp32", autotune=0)
    p0 = train[0]
    coef = [T(a) for a in (p0.bx, p0.by, p0.bz)]
    solver.set_coeffs(*coef)

    def solve(prob, guess):
        p = guess.clone()
        info = solver.solve(T(prob.b), p, tol)
        assert info.status == 0
        return p, info.cycles

    sols = [solve(pr, torch.zeros(pr.cells, device="cuda:0"))[0] for pr in train]
    net = WarmStartNet(dims, seed=0, lr=2e-3)
    for epoch in range(12):
        for t in range(1, len(train)):
            net.train_step(T(train[t].b), *coef, sols[t - 1], sols[t])
    zero_c, net_c, prev_c = [], [], []
    prev = solve(held[0], torch.zeros(held[0].cells, device="cuda:0"))[0]
    for pr in held[1:]:
        z = solve(pr, torch.zeros(pr.cells, device="cuda:0"))
        guess = net.infer(T(pr.b), *coef, prev).clone()
        w = solve(pr, guess)
        zero_c.append(z[1])
        net_c.append(w[1])
        prev_c.append(solve(pr, prev)[1])
        prev = z[0]
    solver.close()
    print("loss first/last", net.loss_history[0], net.loss_history[-1], "V-cycles zero", zero_c, "net", net_c,
          "previous", prev_c)
    assert np.mean(net_c) < np.mean(zero_c), (zero_c, net_c)
