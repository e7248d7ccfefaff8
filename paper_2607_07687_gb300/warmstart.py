"""Learned warm start: a small 3D U-Net that predicts a solve's initial guess.

Inputs per cell: sigma / s, the mean of the cell's six face coefficients, the
previous pressure / s and its residual r = sigma - A p_prev over s (s = RMS of
sigma); output p0 = p_prev + s * net(...), so the network predicts the
increment over the previous pressure (the solution of A dp = r).  The
solver then iterates from p0 to its usual tolerance, so a poor prediction
costs V-cycles but never accuracy.  Architecture (3x3x3 convolutions with
zero padding, ReLU after each): 16-16 | pool | 32-32 | pool | 64-64 | up,
concat | 32-32 | up, concat | 16-16 | 1x1x1 -> 1.

This class only allocates device memory (torch) and sequences the
gmg_net_* kernels of include/gmg_net.h; every arithmetic step runs in them.
Grid dimensions must be multiples of 4 (two 2x poolings).
"""
from __future__ import annotations

import ctypes
import math
from typing import Dict, Optional

import numpy as np

from . import binding as G

# (name, input channels, output channels, level)
LAYERS = [
    ("e0a", 4, 16, 0), ("e0b", 16, 16, 0),
    ("e1a", 16, 32, 1), ("e1b", 32, 32, 1),
    ("e2a", 32, 64, 2), ("e2b", 64, 64, 2),
    ("d1a", 96, 32, 1), ("d1b", 32, 32, 1),
    ("d0a", 48, 16, 0), ("d0b", 16, 16, 0),
]


def _pad16(c: int) -> int:
    return max(16, (c + 15) // 16 * 16)


class _Param:
    """FP32 master values, Adam moments, gradient and BF16 copies of one layer."""

    def __init__(self, torch, dev, n, shape_bf16=None, shape_flip=None):
        self.w = torch.zeros(n, dtype=torch.float32, device=dev)
        self.g = torch.zeros(n, dtype=torch.float32, device=dev)
        self.m = torch.zeros(n, dtype=torch.float32, device=dev)
        self.v = torch.zeros(n, dtype=torch.float32, device=dev)
        self.wb = torch.zeros(shape_bf16, dtype=torch.bfloat16, device=dev) if shape_bf16 else None
        self.wt = torch.zeros(shape_flip, dtype=torch.bfloat16, device=dev) if shape_flip else None


class WarmStartNet:
    def __init__(self, dims, periodic=(False, False, False), seed: int = 0, lr: float = 1e-3, stream=None,
                 loss: str = "mse"):
        import torch
        self.torch = torch
        nx, ny, nz = (int(d) for d in dims)
        if nx % 4 or ny % 4 or nz % 4:
            raise ValueError("grid dimensions must be multiples of 4")
        self.D, self.H, self.W = nz, ny, nx
        self.periodic = tuple(bool(p) for p in periodic)
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.stream = G._stream(stream)
        self.lr = lr
        if loss not in ("mse", "residual"):
            raise ValueError("loss: 'mse' (against the converged pressure) or 'residual' (|b - A p0| / |b|)")
        self.loss_kind = loss
        self.t = 0
        self.loss_history = []
        dev = self.dev
        lv = [(nz, ny, nx), (nz // 2, ny // 2, nx // 2), (nz // 4, ny // 4, nx // 4)]
        self.levels = lv
        self.ncell = [a * b * c for a, b, c in lv]

        def act(level, ch):
            return torch.zeros((self.ncell[level], ch), dtype=torch.bfloat16, device=dev)

        # activations (channels last); c0 / c1 are the decoder's concatenated inputs
        self.a = {"x0": act(0, 16), "e0a": act(0, 16), "c0": act(0, 48), "d0a": act(0, 16), "d0b": act(0, 16),
                  "p1": act(1, 16), "e1a": act(1, 32), "c1": act(1, 96), "d1a": act(1, 32), "d1b": act(1, 32),
                  "p2": act(2, 32), "e2a": act(2, 64), "e2b": act(2, 64)}
        # gradients
        self.gr = {"c0": act(0, 48), "l0a": act(0, 16), "l0b": act(0, 16), "c1": act(1, 96), "l1a": act(1, 32),
                   "l1b": act(1, 32), "p1": act(1, 16), "l2a": act(2, 64), "l2b": act(2, 64), "p2": act(2, 32)}
        self.out = torch.zeros(self.ncell[0], dtype=torch.float32, device=dev)
        self.gout = torch.zeros_like(self.out)
        self.p0 = torch.zeros_like(self.out)
        self.s = torch.zeros(2, dtype=torch.float32, device=dev)   # RMS of sigma, RMS of the residual
        self.red = torch.zeros(4, dtype=torch.float64, device=dev)
        self.loss_dev = torch.zeros(1, dtype=torch.float64, device=dev)
        self.work = torch.zeros(2 * self.ncell[0], dtype=torch.float32, device=dev) if loss == "residual" else None

        # parameters, initialised on the host (He normal, zero biases) and packed
        rng = np.random.default_rng(seed)
        self.params: Dict[str, _Param] = {}
        self.bias: Dict[str, _Param] = {}
        self.ci_pad = {}
        for name, ci, co, _ in LAYERS:
            cp = _pad16(ci)
            self.ci_pad[name] = cp
            w = np.zeros((27, co, cp), dtype=np.float32)
            w[:, :, :ci] = (rng.standard_normal((27, co, ci)) * math.sqrt(2.0 / (27 * ci))).astype(np.float32)
            p = _Param(torch, dev, 27 * co * cp, (27, co, cp), (27, cp, co))
            p.w.copy_(torch.from_numpy(w.ravel()))
            self.params[name] = p
            self.bias[name] = _Param(torch, dev, co)
        # the head starts at zero: an untrained net returns the previous pressure,
        # and training only adds the learned increment
        self.head = _Param(torch, dev, 16)
        self.head_b = _Param(torch, dev, 1)
        # BF16 copies: an Adam step with a zero gradient and lr 0 leaves w unchanged
        for name, _, co, _ in LAYERS:
            p = self.params[name]
            self._adam(p, 1, 0.0, co, self.ci_pad[name])

    # ------------------------------------------------------------------ helpers

    @staticmethod
    def _p(t, ch_offset: int = 0):
        """Device pointer of a tensor, optionally advanced by ch_offset elements."""
        return ctypes.c_void_p(t.data_ptr() + ch_offset * t.element_size())

    def _st(self):
        return ctypes.c_void_p(self.stream)

    def _dims(self, level):
        return self.levels[level]

    def _adam(self, p: _Param, t: int, lr: float, co: int = 0, ci: int = 0):
        G.net_call("gmg_net_adam", p.w.numel(), self._p(p.w), self._p(p.g), self._p(p.m), self._p(p.v), t,
                   float(lr), 0.9, 0.999, 1e-8, self._p(p.wb) if p.wb is not None else None,
                   self._p(p.wt) if p.wt is not None else None, co, ci, self._st())

    # ------------------------------------------------------------------ forward

    def pack(self, b, bx, by, bz, p_prev=None):
        """Network input from the right-hand side (grid units), coefficients, previous pressure."""
        D, H, W = self._dims(0)
        per = (ctypes.c_int * 3)(*[int(v) for v in self.periodic])
        G.net_call("gmg_net_pack_input", D, H, W, self._p(b), self._p(p_prev) if p_prev is not None else None,
                   self._p(bx), self._p(by), self._p(bz), per, self._p(self.a["x0"]), self._p(self.s),
                   self._p(self.red), self._st())

    def forward(self):
        a = self.a
        D0, H0, W0 = self._dims(0)
        D1, H1, W1 = self._dims(1)
        D2, H2, W2 = self._dims(2)
        conv = self._conv_at
        conv("e0a", 0, a["x0"], 16, 0, a["e0a"], 16, 0)
        conv("e0b", 0, a["e0a"], 16, 0, a["c0"], 48, 32)
        G.net_call("gmg_net_pool2", D0, H0, W0, self._p(a["c0"], 32), 48, 16, self._p(a["p1"]), 16, 0, self._st())
        conv("e1a", 1, a["p1"], 16, 0, a["e1a"], 32, 0)
        conv("e1b", 1, a["e1a"], 32, 0, a["c1"], 96, 64)
        G.net_call("gmg_net_pool2", D1, H1, W1, self._p(a["c1"], 64), 96, 32, self._p(a["p2"]), 32, 0, self._st())
        conv("e2a", 2, a["p2"], 32, 0, a["e2a"], 64, 0)
        conv("e2b", 2, a["e2a"], 64, 0, a["e2b"], 64, 0)
        G.net_call("gmg_net_up2", D2, H2, W2, self._p(a["e2b"]), 64, 64, self._p(a["c1"]), 96, 0, self._st())
        conv("d1a", 1, a["c1"], 96, 0, a["d1a"], 32, 0)
        conv("d1b", 1, a["d1a"], 32, 0, a["d1b"], 32, 0)
        G.net_call("gmg_net_up2", D1, H1, W1, self._p(a["d1b"]), 32, 32, self._p(a["c0"]), 48, 0, self._st())
        conv("d0a", 0, a["c0"], 48, 0, a["d0a"], 16, 0)
        conv("d0b", 0, a["d0a"], 16, 0, a["d0b"], 16, 0)
        G.net_call("gmg_net_head", D0, H0, W0, self._p(a["d0b"]), 16, self._p(self.head.w), self._p(self.head_b.w),
                   self._p(self.out), self._st())

    def _conv_at(self, name, level, x, cx, xoff, y, cy, yoff, relu=True):
        _, ci, co, _ = next(l for l in LAYERS if l[0] == name)
        D, H, W = self._dims(level)
        G.net_call("gmg_net_conv3", D, H, W, self._p(x, xoff), cx, self.ci_pad[name], self._p(self.params[name].wb),
                   self._p(self.bias[name].w), co, 1 if relu else 0, self._p(y), cy, yoff, self._st())

    def infer(self, b, bx, by, bz, p_prev=None):
        """Predicted initial guess p0 (FP32 device tensor of the grid's cells)."""
        self.pack(b, bx, by, bz, p_prev)
        self.forward()
        G.net_call("gmg_net_unscale", self.ncell[0], self._p(self.out), self._p(self.s),
                   self._p(p_prev) if p_prev is not None else None, self._p(self.p0), self._st())
        return self.p0

    # ------------------------------------------------------------------ backward

    def _dgrad(self, name, level, g, cg, gx, cgx):
        """Input gradient of layer `name`: the convolution with flipped weights."""
        _, ci, co, _ = next(l for l in LAYERS if l[0] == name)
        D, H, W = self._dims(level)
        G.net_call("gmg_net_conv3", D, H, W, self._p(g), cg, co, self._p(self.params[name].wt), None,
                   self.ci_pad[name], 0, self._p(gx), cgx, 0, self._st())

    def _wgrad(self, name, level, x, cx, xoff, g, cg):
        _, ci, co, _ = next(l for l in LAYERS if l[0] == name)
        D, H, W = self._dims(level)
        G.net_call("gmg_net_conv3_wgrad", D, H, W, self._p(x, xoff), cx, self.ci_pad[name], self._p(g), cg, co,
                   self._p(self.params[name].g), self._p(self.bias[name].g), self._st())

    def _relu_b(self, level, g, cg, y, cy, yoff, C):
        D, H, W = self._dims(level)
        G.net_call("gmg_net_relu_backward", D, H, W, self._p(g), cg, self._p(y, yoff), cy, C, self._st())

    def backward(self):
        """Gradients of every parameter from self.gout (d loss / d out)."""
        a, gr = self.a, self.gr
        D0, H0, W0 = self._dims(0)
        D1, H1, W1 = self._dims(1)
        D2, H2, W2 = self._dims(2)
        for p in list(self.params.values()) + list(self.bias.values()) + [self.head, self.head_b]:
            G.net_call("gmg_net_zero", p.g.numel(), self._p(p.g), self._st())
        G.net_call("gmg_net_head_backward", D0, H0, W0, self._p(self.gout), self._p(a["d0b"]), 16,
                   self._p(self.head.w), self._p(gr["l0b"]), self._p(self.head.g), self._p(self.head_b.g), self._st())
        # level 0 decoder
        self._relu_b(0, gr["l0b"], 16, a["d0b"], 16, 0, 16)
        self._wgrad("d0b", 0, a["d0a"], 16, 0, gr["l0b"], 16)
        self._dgrad("d0b", 0, gr["l0b"], 16, gr["l0a"], 16)
        self._relu_b(0, gr["l0a"], 16, a["d0a"], 16, 0, 16)
        self._wgrad("d0a", 0, a["c0"], 48, 0, gr["l0a"], 16)
        self._dgrad("d0a", 0, gr["l0a"], 16, gr["c0"], 48)
        G.net_call("gmg_net_up2_backward", D1, H1, W1, self._p(gr["c0"]), 48, 0, 32, self._p(gr["l1b"]), 32, self._st())
        # level 1 decoder
        self._relu_b(1, gr["l1b"], 32, a["d1b"], 32, 0, 32)
        self._wgrad("d1b", 1, a["d1a"], 32, 0, gr["l1b"], 32)
        self._dgrad("d1b", 1, gr["l1b"], 32, gr["l1a"], 32)
        self._relu_b(1, gr["l1a"], 32, a["d1a"], 32, 0, 32)
        self._wgrad("d1a", 1, a["c1"], 96, 0, gr["l1a"], 32)
        self._dgrad("d1a", 1, gr["l1a"], 32, gr["c1"], 96)
        G.net_call("gmg_net_up2_backward", D2, H2, W2, self._p(gr["c1"]), 96, 0, 64, self._p(gr["l2b"]), 64, self._st())
        # level 2
        self._relu_b(2, gr["l2b"], 64, a["e2b"], 64, 0, 64)
        self._wgrad("e2b", 2, a["e2a"], 64, 0, gr["l2b"], 64)
        self._dgrad("e2b", 2, gr["l2b"], 64, gr["l2a"], 64)
        self._relu_b(2, gr["l2a"], 64, a["e2a"], 64, 0, 64)
        self._wgrad("e2a", 2, a["p2"], 32, 0, gr["l2a"], 64)
        self._dgrad("e2a", 2, gr["l2a"], 64, gr["p2"], 32)
        # level 1 encoder: pooled gradient plus the skip connection's
        G.net_call("gmg_net_pool2_backward", D1, H1, W1, self._p(gr["p2"]), 32, 32, self._p(gr["l1b"]), 32,
                   self._p(gr["c1"]), 96, 64, self._st())
        self._relu_b(1, gr["l1b"], 32, a["c1"], 96, 64, 32)
        self._wgrad("e1b", 1, a["e1a"], 32, 0, gr["l1b"], 32)
        self._dgrad("e1b", 1, gr["l1b"], 32, gr["l1a"], 32)
        self._relu_b(1, gr["l1a"], 32, a["e1a"], 32, 0, 32)
        self._wgrad("e1a", 1, a["p1"], 16, 0, gr["l1a"], 32)
        self._dgrad("e1a", 1, gr["l1a"], 32, gr["p1"], 16)
        # level 0 encoder
        G.net_call("gmg_net_pool2_backward", D0, H0, W0, self._p(gr["p1"]), 16, 16, self._p(gr["l0b"]), 16,
                   self._p(gr["c0"]), 48, 32, self._st())
        self._relu_b(0, gr["l0b"], 16, a["c0"], 48, 32, 16)
        self._wgrad("e0b", 0, a["e0a"], 16, 0, gr["l0b"], 16)
        self._dgrad("e0b", 0, gr["l0b"], 16, gr["l0a"], 16)
        self._relu_b(0, gr["l0a"], 16, a["e0a"], 16, 0, 16)
        self._wgrad("e0a", 0, a["x0"], 16, 0, gr["l0a"], 16)

    def loss(self, p_target, p_prev=None):
        """Loss of the prediction against the converged pressure (d loss / d out in self.gout)."""
        D, H, W = self._dims(0)
        G.net_call("gmg_net_loss", D, H, W, self._p(self.out), self._p(p_target),
                   self._p(p_prev) if p_prev is not None else None, self._p(self.s),
                   self._p(self.gout), self._p(self.loss_dev), self._p(self.red), self._st())

    def residual_loss(self, b, bx, by, bz, p_prev=None):
        """Squared relative residual |b - A p0|^2 / |b|^2 of the prediction (d loss / d out in self.gout)."""
        D, H, W = self._dims(0)
        if self.work is None:
            self.work = self.torch.zeros(2 * self.ncell[0], dtype=self.torch.float32, device=self.dev)
        per = (ctypes.c_int * 3)(*[int(v) for v in self.periodic])
        G.net_call("gmg_net_residual_loss", D, H, W, self._p(self.out),
                   self._p(p_prev) if p_prev is not None else None, self._p(self.s), self._p(b), self._p(bx),
                   self._p(by), self._p(bz), per, self._p(self.work), self._p(self.gout), self._p(self.loss_dev),
                   self._p(self.red), self._st())

    def step(self):
        """One Adam update of every parameter."""
        self.t += 1
        for name, _, co, _ in LAYERS:
            self._adam(self.params[name], self.t, self.lr, co, self.ci_pad[name])
            self._adam(self.bias[name], self.t, self.lr)
        self._adam(self.head, self.t, self.lr)
        self._adam(self.head_b, self.t, self.lr)

    def train_step(self, b, bx, by, bz, p_prev, p_target=None) -> float:
        """Forward, loss, backward and Adam on one input (and its converged pressure for the MSE loss)."""
        self.pack(b, bx, by, bz, p_prev)
        self.forward()
        if self.loss_kind == "residual":
            self.residual_loss(b, bx, by, bz, p_prev)
        else:
            self.loss(p_target, p_prev)
        self.backward()
        self.step()
        loss = float(self.loss_dev.item())
        self.loss_history.append(loss)
        return loss

    # ------------------------------------------------------------------ parameters

    def state_dict(self):
        sd = {}
        for name in self.params:
            sd[name + ".w"] = self.params[name].w.detach().cpu().clone()
            sd[name + ".b"] = self.bias[name].w.detach().cpu().clone()
        sd["out.w"] = self.head.w.detach().cpu().clone()
        sd["out.b"] = self.head_b.w.detach().cpu().clone()
        return sd

    def load_state_dict(self, sd):
        for name, _, co, _ in LAYERS:
            self.params[name].w.copy_(sd[name + ".w"].to(self.dev))
            self.bias[name].w.copy_(sd[name + ".b"].to(self.dev))
            self._adam(self.params[name], 1, 0.0, co, self.ci_pad[name])
        self.head.w.copy_(sd["out.w"].to(self.dev))
        self.head_b.w.copy_(sd["out.b"].to(self.dev))

    def set_weights(self, params):
        """Load weights given in the logical layout: "<layer>.w" [co][ci][3][3][3],
        "<layer>.b" [co], "out.w" [1][16], "out.b" [1] (host arrays)."""
        torch = self.torch
        for name, ci, co, _ in LAYERS:
            cp = self.ci_pad[name]
            w = np.zeros((27, co, cp), dtype=np.float32)
            w[:, :, :ci] = np.asarray(params[name + ".w"], dtype=np.float64).reshape(co, ci, 27).transpose(2, 0, 1)
            self.params[name].w.copy_(torch.from_numpy(w.ravel()))
            self.bias[name].w.copy_(torch.from_numpy(np.asarray(params[name + ".b"], dtype=np.float32)))
            self._adam(self.params[name], 1, 0.0, co, cp)
        self.head.w.copy_(torch.from_numpy(np.asarray(params["out.w"], dtype=np.float32).reshape(16)))
        self.head_b.w.copy_(torch.from_numpy(np.asarray(params["out.b"], dtype=np.float32).reshape(1)))

    def _logical(self, name, flat):
        _, ci, co, _ = next(l for l in LAYERS if l[0] == name)
        w = flat.detach().cpu().numpy().astype(np.float64).reshape(27, co, self.ci_pad[name])[:, :, :ci]
        return np.ascontiguousarray(w.transpose(1, 2, 0).reshape(co, ci, 3, 3, 3))

    def weights(self):
        """Master weights (FP32 values) in the logical layout of set_weights."""
        out = {}
        for name, _, _, _ in LAYERS:
            out[name + ".w"] = self._logical(name, self.params[name].w)
            out[name + ".b"] = self.bias[name].w.detach().cpu().numpy().astype(np.float64)
        out["out.w"] = self.head.w.detach().cpu().numpy().astype(np.float64).reshape(1, 16)
        out["out.b"] = self.head_b.w.detach().cpu().numpy().astype(np.float64)
        return out

    def gradients(self):
        """Gradients of the last backward() in the logical layout of set_weights."""
        out = {}
        for name, _, _, _ in LAYERS:
            out[name + ".w"] = self._logical(name, self.params[name].g)
            out[name + ".b"] = self.bias[name].g.detach().cpu().numpy().astype(np.float64)
        out["out.w"] = self.head.g.detach().cpu().numpy().astype(np.float64).reshape(1, 16)
        out["out.b"] = self.head_b.g.detach().cpu().numpy().astype(np.float64)
        return out
