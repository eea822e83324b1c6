"""FP64 reference of the surrogate network (test infrastructure only).

A plain numpy statement of the convolutional U-Net the CUDA surrogate runs:
forward and backward of every layer written from their definitions
(3 x 3 same-padded convolution as a sum of nine shifted products, ReLU, 2 x 2
max pooling, 2 x 2 stride-2 up-convolution, channel concatenation, 1 x 1
output projection with a residual connection, mean squared error).  Only the
tests and the smoke check import it; it shares no code with the CUDA path.

Layouts (shared by definition with the CUDA network, not by code):
  activations NHWC [B, H, W, C];
  conv3x3 weight [Cout, 9 * Cin], column (ky * 3 + kx) * Cin + ci, bias [Cout];
  up-convolution weight [4 * Cout, Cin], row (dy * 2 + dx) * Cout + co,
    bias [4 * Cout] (one per sub-pixel and channel);
  projection weight [O, C], bias [O].
Network with L levels and base width w: level l has width w * 2**l; encoder
level l: two conv3x3 + ReLU, then (l < L - 1) 2 x 2 max pooling; decoder level
l = L-2 .. 0: up-convolution of the level below, concatenation [skip, up],
two conv3x3 + ReLU; output = x[..., :O] + projection of the top decoder
level.

Rounding points.  `forward` and `backward` take an optional quantiser q
(default: none, pure FP64).  With q = bf16_round they round where a BF16
network stores values: every convolution and up-convolution output, and every
activation gradient that a BF16 GEMM consumes (after its ReLU mask).  The
arithmetic between those points stays FP64.  This matters for comparisons:
a ReLU whose pre-activation lies within rounding distance of zero switches
between the two evaluations, and a fraction f of switched units moves a
weight gradient by about sqrt(f) in relative terms, far more than the
rounding itself.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, W, b):
    B, H, Wd, Ci = x.shape
    Co = W.shape[0]
    Wt = W.reshape(Co, 3, 3, Ci)
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.broadcast_to(b, (B, H, Wd, Co)).copy()
    for ky in range(3):
        for kx in range(3):
            y += xp[:, ky:ky + H, kx:kx + Wd, :] @ Wt[:, ky, kx, :].T
    return y


def conv3x3_bwd(x, W, dy):
    B, H, Wd, Ci = x.shape
    Co = W.shape[0]
    Wt = W.reshape(Co, 3, 3, Ci)
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dW = np.zeros((Co, 3, 3, Ci))
    for ky in range(3):
        for kx in range(3):
            xs = xp[:, ky:ky + H, kx:kx + Wd, :]
            dW[:, ky, kx, :] = np.einsum("bhwo,bhwi->oi", dy, xs)
            dxp[:, ky:ky + H, kx:kx + Wd, :] += dy @ Wt[:, ky, kx, :]
    return dxp[:, 1:-1, 1:-1, :], dW.reshape(Co, 9 * Ci), dy.sum(axis=(0, 1, 2))


def maxpool(x):
    B, H, W, C = x.shape
    v = x.reshape(B, H // 2, 2, W // 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(B, H // 2, W // 2, 4, C)
    arg = v.argmax(axis=3)  # first maximum in (dy, dx) row-major order
    return np.take_along_axis(v, arg[:, :, :, None, :], axis=3)[:, :, :, 0, :], arg


def maxpool_bwd(dy, arg, shape):
    B, H, W, C = shape
    g = np.zeros((B, H // 2, W // 2, 4, C))
    np.put_along_axis(g, arg[:, :, :, None, :], dy[:, :, :, None, :], axis=3)
    return g.reshape(B, H // 2, W // 2, 2, 2, C).transpose(0, 1, 3, 2, 4, 5).reshape(B, H, W, C)


def upconv(x, W, b):
    B, H, Wd, Ci = x.shape
    Co = W.shape[0] // 4
    u = (x @ W.T + b).reshape(B, H, Wd, 2, 2, Co)
    return u.transpose(0, 1, 3, 2, 4, 5).reshape(B, 2 * H, 2 * Wd, Co)


def upconv_bwd(x, W, dy):
    B, H, Wd, Ci = x.shape
    Co = W.shape[0] // 4
    du = dy.reshape(B, H, 2, Wd, 2, Co).transpose(0, 1, 3, 2, 4, 5).reshape(B, H, Wd, 4 * Co)
    dx = du @ W
    dW = np.einsum("bhwk,bhwi->ki", du, x)
    db = du.sum(axis=(0, 1, 2))
    return dx, dW, db


def relu(x):
    return np.maximum(x, 0.0)


def bf16_round(a):
    """Nearest BF16 value (ties to even) of each element, as FP64: the FP64
    value is first rounded to FP32, then its 32-bit pattern is rounded to the
    upper 16 bits."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = ((b + 0x7FFF + lsb) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64).reshape(np.shape(a))


def _ident(a):
    return a


def init_shapes(levels: int, base: int, in_ch: int, out_ch: int):
    """Parameter names and shapes of the network, in a fixed order."""
    shapes = []
    c_prev = in_ch
    for l in range(levels):
        c = base * 2**l
        shapes += [(f"enc{l}a.W", (c, 9 * c_prev)), (f"enc{l}a.b", (c,)),
                   (f"enc{l}b.W", (c, 9 * c)), (f"enc{l}b.b", (c,))]
        c_prev = c
    for l in range(levels - 2, -1, -1):
        c = base * 2**l
        shapes += [(f"up{l}.W", (4 * c, 2 * c)), (f"up{l}.b", (4 * c,)),
                   (f"dec{l}a.W", (c, 9 * 2 * c)), (f"dec{l}a.b", (c,)),
                   (f"dec{l}b.W", (c, 9 * c)), (f"dec{l}b.b", (c,))]
    shapes += [("out.W", (out_ch, base)), ("out.b", (out_ch,))]
    return shapes


def forward(params: dict, x, levels: int, out_ch: int, q=None):
    """y = x[..., :out_ch] + projection; returns y and the cache of activations."""
    q = q or _ident
    cache = {"x": x}
    h = x
    for l in range(levels):
        a = q(relu(conv3x3(h, params[f"enc{l}a.W"], params[f"enc{l}a.b"])))
        s = q(relu(conv3x3(a, params[f"enc{l}b.W"], params[f"enc{l}b.b"])))
        cache[f"enc{l}.in"], cache[f"enc{l}.a"], cache[f"enc{l}.s"] = h, a, s
        if l < levels - 1:
            h, cache[f"pool{l}.arg"] = maxpool(s)
        else:
            h = s
    for l in range(levels - 2, -1, -1):
        u = q(upconv(h, params[f"up{l}.W"], params[f"up{l}.b"]))
        cat = np.concatenate([cache[f"enc{l}.s"], u], axis=3)
        a = q(relu(conv3x3(cat, params[f"dec{l}a.W"], params[f"dec{l}a.b"])))
        d = q(relu(conv3x3(a, params[f"dec{l}b.W"], params[f"dec{l}b.b"])))
        cache[f"up{l}.in"], cache[f"dec{l}.cat"], cache[f"dec{l}.a"], cache[f"dec{l}.d"] = h, cat, a, d
        h = d
    cache["top"] = h
    y = x[..., :out_ch] + h @ params["out.W"].T + params["out.b"]
    return y, cache


def backward(params: dict, cache: dict, dy, levels: int, q=None):
    """Gradients of every parameter for the output gradient dy."""
    q = q or _ident
    g = {}
    top = cache["top"]
    g["out.W"] = np.einsum("bhwo,bhwc->oc", dy, top)
    g["out.b"] = dy.sum(axis=(0, 1, 2))
    dh = dy @ params["out.W"]
    skip_grad = {}
    for l in range(0, levels - 1):
        dd = q(dh * (cache[f"dec{l}.d"] > 0))
        da, g[f"dec{l}b.W"], g[f"dec{l}b.b"] = conv3x3_bwd(cache[f"dec{l}.a"], params[f"dec{l}b.W"], dd)
        da = q(da * (cache[f"dec{l}.a"] > 0))
        dcat, g[f"dec{l}a.W"], g[f"dec{l}a.b"] = conv3x3_bwd(cache[f"dec{l}.cat"], params[f"dec{l}a.W"], da)
        c = params[f"dec{l}b.W"].shape[0]
        skip_grad[l] = dcat[..., :c]
        dh, g[f"up{l}.W"], g[f"up{l}.b"] = upconv_bwd(cache[f"up{l}.in"], params[f"up{l}.W"], q(dcat[..., c:]))
    for l in range(levels - 1, -1, -1):
        ds = dh if l == levels - 1 else skip_grad[l] + maxpool_bwd(dh, cache[f"pool{l}.arg"], cache[f"enc{l}.s"].shape)
        ds = q(ds * (cache[f"enc{l}.s"] > 0))
        da, g[f"enc{l}b.W"], g[f"enc{l}b.b"] = conv3x3_bwd(cache[f"enc{l}.a"], params[f"enc{l}b.W"], ds)
        da = q(da * (cache[f"enc{l}.a"] > 0))
        dh, g[f"enc{l}a.W"], g[f"enc{l}a.b"] = conv3x3_bwd(cache[f"enc{l}.in"], params[f"enc{l}a.W"], da)
    return g


def mse(y, t, x=None, alpha=0.0):
    """Mean squared error and its gradient; with the input x (fields last,
    phase field first), each pixel's squared errors weighted by
    w = 1 + alpha max(0, 1 - phi^2): mean(w d^2), gradient 2 w d / n."""
    d = y - t
    w = 1.0 if x is None else (1.0 + alpha * np.maximum(0.0, 1.0 - x[..., :1] ** 2))
    return float((w * d * d).mean()), 2.0 * w * d / d.size
