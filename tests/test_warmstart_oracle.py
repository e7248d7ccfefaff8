"""Pins of the FP64 warm-start network oracle against facts outside it:
scipy's correlation, adjoint identities, finite differences and the closed
form of Adam's first step."""
import numpy as np
import pytest

from oracle import warmstart_oracle as W


def test_conv3_equals_scipy_correlate():
    import scipy.signal
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 5, 6, 7))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    y = W.conv3(x, w, b)
    for o in range(4):
        ref = b[o] + sum(scipy.signal.correlate(x[i], w[o, i], mode="same", method="direct") for i in range(3))
        np.testing.assert_allclose(y[o], ref, atol=1e-12)


def test_conv3_backward_is_the_adjoint():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5, 6))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    gy = rng.standard_normal((2, 4, 5, 6))
    gx, gw, gb = W.conv3_backward(x, w, gy)
    lhs = float(np.sum((W.conv3(x, w, np.zeros(2))) * gy))
    assert lhs == pytest.approx(float(np.sum(x * gx)), rel=1e-12)
    assert lhs == pytest.approx(float(np.sum(w * gw)), rel=1e-12)
    np.testing.assert_allclose(gb, gy.sum(axis=(1, 2, 3)))


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 4, 6, 8))
    g = rng.standard_normal((2, 2, 3, 4))
    assert float(np.sum(W.pool2(x) * g)) == pytest.approx(float(np.sum(x * W.pool2_backward(g))), rel=1e-12)
    xs = rng.standard_normal((2, 2, 3, 4))
    gs = rng.standard_normal((2, 4, 6, 8))
    assert float(np.sum(W.up2(xs) * gs)) == pytest.approx(float(np.sum(xs * W.up2_backward(gs))), rel=1e-12)
    np.testing.assert_allclose(W.pool2(W.up2(xs)), xs)


def test_loss_gradient_finite_differences():
    rng = np.random.default_rng(3)
    p0 = rng.standard_normal((4, 4, 4))
    pt = rng.standard_normal((4, 4, 4))
    loss, g = W.loss_and_grad_out(p0, pt)
    d = rng.standard_normal(p0.shape)
    eps = 1e-6
    fd = (W.loss_and_grad_out(p0 + eps * d, pt)[0] - W.loss_and_grad_out(p0 - eps * d, pt)[0]) / (2 * eps)
    assert float(np.sum(g * d)) == pytest.approx(fd, rel=1e-7)
    # invariant to shifts of p0
    assert W.loss_and_grad_out(p0 + 3.0, pt)[0] == pytest.approx(loss, rel=1e-12)


def test_network_gradient_finite_differences():
    """Every parameter group of the whole network against central differences
    along a random direction (8^3 grid, FP64)."""
    rng = np.random.default_rng(4)
    params = W.init_params(5)
    for k in params:
        if k.endswith(".b"):
            params[k] = rng.standard_normal(params[k].shape) * 0.1
    x0 = rng.standard_normal((4, 8, 8, 8))
    pt = rng.standard_normal((8, 8, 8))

    def f(p):
        out, _ = W.forward(p, x0)
        return W.loss_and_grad_out(out, pt)[0]

    out, cache = W.forward(params, x0)
    _, gout = W.loss_and_grad_out(out, pt)
    grads = W.backward(params, cache, gout)
    assert set(grads) == set(params)
    for k in sorted(params):
        d = rng.standard_normal(params[k].shape)
        an = float(np.sum(grads[k] * d))
        errs = []
        for eps in (1e-7, 3e-8):       # a kink crossing spoils at most one of the two steps
            pp = dict(params)
            pm = dict(params)
            pp[k] = params[k] + eps * d
            pm[k] = params[k] - eps * d
            fd = (f(pp) - f(pm)) / (2 * eps)
            errs.append(abs(an - fd) / max(abs(fd), 1e-9))
        assert min(errs) <= 1e-5, (k, errs)


def test_adam_first_step_closed_form():
    """After one step m_hat = g and v_hat = g^2: theta moves by lr g / (|g| + eps)."""
    params = {"a": np.array([1.0, -2.0, 0.5])}
    grads = {"a": np.array([0.3, -4.0, 1e-3])}
    state = {}
    W.adam_step(params, grads, state, lr=0.01)
    np.testing.assert_allclose(params["a"], np.array([1.0, -2.0, 0.5]) - 0.01 * grads["a"] / (np.abs(grads["a"]) + 1e-8),
                               rtol=1e-12)


def test_predict_increment_map():
    """p0 = p_prev + s * net: a zeroed network returns p_prev exactly, s is the
    RMS of b, and the parameter gradient of loss(p0) is backward(s * d loss /
    d p0), checked by central differences on one weight tensor."""
    rng = np.random.default_rng(6)
    shape = (8, 8, 8)
    b = rng.standard_normal(shape)
    bm = rng.uniform(0, 1, shape)
    pp = rng.standard_normal(shape)
    r = 0.01 * rng.standard_normal(shape)
    pt = pp + 0.3 * rng.standard_normal(shape)
    params = W.init_params(7)
    zero = {k: np.zeros_like(v) for k, v in params.items()}
    p0, _, s = W.predict(zero, b, bm, pp, r)
    assert np.array_equal(p0, pp) and s == pytest.approx(np.sqrt(np.mean(b * b)))
    x0, s = W.features(b, bm, pp, r)
    np.testing.assert_allclose(x0[3] * s, r)
    np.testing.assert_allclose(x0[2] * s, pp)
    p0, cache, s = W.predict(params, b, bm, pp, r)
    _, g = W.loss_and_grad_out(p0, pt)
    grads = W.backward(params, cache, s * g)
    d = rng.standard_normal(params["d1a.w"].shape)

    def f(w):
        q = dict(params)
        q["d1a.w"] = w
        return W.loss_and_grad_out(W.predict(q, b, bm, pp, r)[0], pt)[0]
    errs = []
    for eps in (1e-7, 3e-8):
        fd = (f(params["d1a.w"] + eps * d) - f(params["d1a.w"] - eps * d)) / (2 * eps)
        errs.append(abs(float(np.sum(grads["d1a.w"] * d)) - fd) / abs(fd))
    assert min(errs) <= 1e-5, errs


def test_residual_loss_gradient(oracle):
    """The residual loss's gradient: central differences, and equality with
    -2 A^T r / |b|^2 from the dense assembly of the operator (A^T = A)."""
    rng = np.random.default_rng(8)
    shape = (4, 4, 6)
    per = (False, True, False)
    bx, by, bz = (rng.uniform(0.1, 1.0, shape) for _ in range(3))
    A = lambda v: oracle.apply_A(v, bx, by, bz, periodic=per)
    b = rng.standard_normal(shape)
    p0 = rng.standard_normal(shape)
    loss, g = W.residual_loss_and_grad(p0, b, A)
    M = oracle.dense_operator(bx, by, bz, periodic=per)
    r = b.ravel() - M @ p0.ravel()
    np.testing.assert_allclose(loss, r @ r / (b.ravel() @ b.ravel()), rtol=1e-12)
    np.testing.assert_allclose(g.ravel(), -2.0 * M.T @ r / (b.ravel() @ b.ravel()), rtol=1e-10, atol=1e-14)
    d = rng.standard_normal(shape)
    eps = 1e-6
    fd = (W.residual_loss_and_grad(p0 + eps * d, b, A)[0] - W.residual_loss_and_grad(p0 - eps * d, b, A)[0]) / (2 * eps)
    assert float(np.sum(g * d)) == pytest.approx(fd, rel=1e-7)
