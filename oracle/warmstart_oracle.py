"""FP64 CPU oracle of the learned warm-start network.

TEST INFRASTRUCTURE ONLY: the tests and the smoke check use it; the solver
package never imports it.

The network predicts the initial guess p0 of a pressure-Poisson solve from
(sigma, mean face coefficient, previous pressure, residual of the previous
pressure).  It is a small 3-level
U-Net of 3x3x3 convolutions (16 / 32 / 64 channels) with 2x average pooling,
nearest 2x upsampling and channel concatenation of the encoder features,
finished by a 1x1x1 convolution.  Everything here is written from the
definitions, in FP64, on arrays laid out [C][D][H][W] (z, y, x):

    conv:     y[o, z, y, x] = b[o] + sum_{i, a, b, c} W[o, i, a, b, c] x[i, z+a-1, y+b-1, x+c-1]
              (zero outside the grid)
    relu:     max(v, 0)
    pool:     mean of each 2 x 2 x 2 block
    upsample: each value copied to its 2 x 2 x 2 block
    input:    x0 = (b / s, mean face coefficient, p_prev / s, r / s) with
              r = b - A p_prev and s = RMS(b)
    output:   p0 = p_prev + s * net(x0)  (the net predicts the increment over
              the previous pressure, which solves A dp = r, in units of s)
    loss:     |(p0 - mean p0) - (p* - mean p*)|^2 / |p* - mean p*|^2, or the
              squared relative residual |b - A p0|^2 / |b|^2 (the quantity the
              solver's stopping test measures)

Backward passes are the adjoints of these maps, written out term by term.
"""
from __future__ import annotations

import numpy as np

# (name, input channels, output channels, level)
LAYERS = [
    ("e0a", 4, 16, 0), ("e0b", 16, 16, 0),
    ("e1a", 16, 32, 1), ("e1b", 32, 32, 1),
    ("e2a", 32, 64, 2), ("e2b", 64, 64, 2),
    ("d1a", 96, 32, 1), ("d1b", 32, 32, 1),
    ("d0a", 48, 16, 0), ("d0b", 16, 16, 0),
]
OUT = ("out", 16, 1)


def init_params(seed: int = 0):
    """He-initialised weights (FP64); zero biases."""
    rng = np.random.default_rng(seed)
    params = {}
    for name, ci, co, _ in LAYERS:
        params[name + ".w"] = rng.standard_normal((co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci))
        params[name + ".b"] = np.zeros(co)
    params["out.w"] = rng.standard_normal((1, 16)) * np.sqrt(1.0 / 16)
    params["out.b"] = np.zeros(1)
    return params


def _pad(x):
    return np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))


def conv3(x, w, b):
    """3x3x3 convolution with zero padding; x [Ci][D][H][W], w [Co][Ci][3][3][3]."""
    ci, d, h, wd = x.shape
    xp = _pad(x)
    y = np.zeros((w.shape[0], d, h, wd))
    for a in range(3):
        for bb in range(3):
            for c in range(3):
                win = xp[:, a:a + d, bb:bb + h, c:c + wd]
                y += np.einsum("oi,izyx->ozyx", w[:, :, a, bb, c], win)
    return y + b[:, None, None, None]


def conv3_backward(x, w, gy):
    """Gradients of conv3 w.r.t. x, w and b for the output gradient gy."""
    ci, d, h, wd = x.shape
    xp = _pad(x)
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for a in range(3):
        for bb in range(3):
            for c in range(3):
                win = xp[:, a:a + d, bb:bb + h, c:c + wd]
                gw[:, :, a, bb, c] = np.einsum("ozyx,izyx->oi", gy, win)
                gxp[:, a:a + d, bb:bb + h, c:c + wd] += np.einsum("oi,ozyx->izyx", w[:, :, a, bb, c], gy)
    gb = gy.sum(axis=(1, 2, 3))
    return gxp[:, 1:-1, 1:-1, 1:-1], gw, gb


def relu(v):
    return np.maximum(v, 0.0)


def pool2(x):
    c, d, h, w = x.shape
    return x.reshape(c, d // 2, 2, h // 2, 2, w // 2, 2).mean(axis=(2, 4, 6))


def pool2_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up2_backward(g):
    c, d, h, w = g.shape
    return g.reshape(c, d // 2, 2, h // 2, 2, w // 2, 2).sum(axis=(2, 4, 6))


def forward(params, x0):
    """x0 [4][D][H][W] -> (out [D][H][W], cache of activations)."""
    cache = {"x0": x0}
    h = x0
    for name in ("e0a", "e0b"):
        h = relu(conv3(h, params[name + ".w"], params[name + ".b"]))
        cache[name] = h
    h = pool2(h)
    cache["p1"] = h
    for name in ("e1a", "e1b"):
        h = relu(conv3(h, params[name + ".w"], params[name + ".b"]))
        cache[name] = h
    h = pool2(h)
    cache["p2"] = h
    for name in ("e2a", "e2b"):
        h = relu(conv3(h, params[name + ".w"], params[name + ".b"]))
        cache[name] = h
    h = np.concatenate([up2(h), cache["e1b"]], axis=0)
    cache["c1"] = h
    for name in ("d1a", "d1b"):
        h = relu(conv3(h, params[name + ".w"], params[name + ".b"]))
        cache[name] = h
    h = np.concatenate([up2(h), cache["e0b"]], axis=0)
    cache["c0"] = h
    for name in ("d0a", "d0b"):
        h = relu(conv3(h, params[name + ".w"], params[name + ".b"]))
        cache[name] = h
    out = np.einsum("oi,izyx->ozyx", params["out.w"], h)[0] + params["out.b"][0]
    return out, cache


def loss_and_grad_out(p0, ptarget):
    """Normalised zero-mean MSE and its gradient w.r.t. p0."""
    a = p0 - p0.mean()
    t = ptarget - ptarget.mean()
    den = float(np.sum(t * t))
    diff = a - t
    loss = float(np.sum(diff * diff)) / den
    g = 2.0 * diff / den
    return loss, g - g.mean()


def residual_loss_and_grad(p0, b, apply_A):
    """|b - A p0|^2 / |b|^2 and its gradient -2 A^T (b - A p0) / |b|^2 w.r.t. p0.
    apply_A is the (symmetric) operator; A^T = A."""
    r = b - apply_A(p0)
    den = float(np.sum(b * b))
    return float(np.sum(r * r)) / den, -2.0 * apply_A(r) / den


def backward(params, cache, gout, record=None):
    """Gradients of every parameter for d(loss)/d(out) = gout [D][H][W].  If record
    is a dict, it receives each layer's output gradient after the ReLU mask (the
    g its weight gradient sums against the layer's input)."""
    grads = {}
    h = cache["d0b"]
    grads["out.w"] = np.einsum("zyx,izyx->i", gout, h)[None, :]
    grads["out.b"] = np.array([gout.sum()])
    g = params["out.w"][0][:, None, None, None] * gout[None]

    def layer(name, inp, g):
        g = g * (cache[name] > 0)
        if record is not None:
            record[name] = g
        gx, gw, gb = conv3_backward(inp, params[name + ".w"], g)
        grads[name + ".w"] = gw
        grads[name + ".b"] = gb
        return gx

    g = layer("d0b", cache["d0a"], g)
    g = layer("d0a", cache["c0"], g)
    c_up = cache["d1b"].shape[0]
    g_up, g_e0 = g[:c_up], g[c_up:]
    g = up2_backward(g_up)
    g = layer("d1b", cache["d1a"], g)
    g = layer("d1a", cache["c1"], g)
    c_up = cache["e2b"].shape[0]
    g_up, g_e1 = g[:c_up], g[c_up:]
    g = up2_backward(g_up)
    g = layer("e2b", cache["e2a"], g)
    g = layer("e2a", cache["p2"], g)
    g = pool2_backward(g) + g_e1
    g = layer("e1b", cache["e1a"], g)
    g = layer("e1a", cache["p1"], g)
    g = pool2_backward(g) + g_e0
    g = layer("e0b", cache["e0a"], g)
    layer("e0a", cache["x0"], g)
    return grads


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (in place); state holds m, v and the step count t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k, g in grads.items():
        m = state.setdefault("m." + k, np.zeros_like(g))
        v = state.setdefault("v." + k, np.zeros_like(g))
        m[...] = b1 * m + (1 - b1) * g
        v[...] = b2 * v + (1 - b2) * g * g
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)


def predict(params, b, beta_mean, p_prev, r):
    """Initial guess p0 = p_prev + s * net(x0), with the network's cache and s."""
    x0, s = features(b, beta_mean, p_prev, r)
    out, cache = forward(params, x0)
    return p_prev + s * out, cache, s


def features(b, beta_mean, p_prev, r):
    """Network input [4][D][H][W] and the scale s = RMS(b) (1 if b = 0)."""
    s = float(np.sqrt(np.mean(b * b)))
    s = s if s > 0 else 1.0
    return np.stack([b / s, beta_mean, p_prev / s, r / s]), s
