"""Binding of the surrogate network (``lbm_unet_*`` in ``include/lbm.h``).

Argument marshalling only: the forward pass, the loss, the backward pass and
the Adam update all run in the library's CUDA kernels.  Tensors passed in are
CUDA ``torch.float32`` arrays of shape [batch, height, width, fields]; torch is
used for device memory and streams only.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import lbm as L

# The network the surrogate runs: five levels of widths 32 .. 512 and five
# fields (phi, C, theta, u_x, u_y) in and out.
LEVELS = 5
BASE = 32
FIELDS = ("phi", "C", "theta", "ux", "uy")
IN_PITCH = 8  # input channels as the first convolution sees them (fields, zero padded)


def param_shapes(levels: int = LEVELS, base: int = BASE, fields: int = len(FIELDS)):
    """(name, shape) of every parameter tensor, in the library's order."""
    shapes = []
    c_prev = IN_PITCH
    for l in range(levels):
        c = base << l
        shapes += [(f"enc{l}a.W", (c, 9 * c_prev)), (f"enc{l}a.b", (c,)),
                   (f"enc{l}b.W", (c, 9 * c)), (f"enc{l}b.b", (c,))]
        c_prev = c
    for l in range(levels - 2, -1, -1):
        c = base << l
        shapes += [(f"up{l}.W", (4 * c, 2 * c)), (f"up{l}.b", (4 * c,)),
                   (f"dec{l}a.W", (c, 18 * c)), (f"dec{l}a.b", (c,)),
                   (f"dec{l}b.W", (c, 9 * c)), (f"dec{l}b.b", (c,))]
    shapes += [("out.W", (fields, base)), ("out.b", (fields,))]
    return shapes


def flatten(params: dict, shapes) -> np.ndarray:
    return np.concatenate([np.asarray(params[n], np.float32).reshape(-1) for n, _ in shapes])


def unflatten(vec: np.ndarray, shapes) -> dict:
    out, o = {}, 0
    for n, shp in shapes:
        k = int(np.prod(shp))
        out[n] = vec[o:o + k].reshape(shp)
        o += k
    return out


class UNet:
    """The network sized for `batch` images of height x width pixels."""

    def __init__(self, batch: int, height: int, width: int, levels: int = LEVELS, base: int = BASE,
                 fields: int = len(FIELDS), stream=None):
        self.lib = L.load()
        h = ct.c_void_p()
        rc = self.lib.lbm_unet_create(levels, base, fields, batch, height, width, ct.byref(h))
        if rc != L.LBM_OK:
            raise L.LBMError(rc, f"lbm_unet_create({levels}, {base}, {fields}, {batch}, {height}, {width})")
        self.h = h
        self.levels, self.base, self.fields = levels, base, fields
        self.shape = (batch, height, width, fields)
        self.shapes = param_shapes(levels, base, fields)
        if stream is not None:
            self.set_stream(stream)

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h:
            self.lib.lbm_unet_destroy(h)

    def _check(self, rc: int) -> None:
        if rc != L.LBM_OK:
            raise L.LBMError(rc, (self.lib.lbm_unet_last_error(self.h) or b"").decode())

    def _t(self, t):
        import torch

        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous(), "CUDA float32 contiguous expected"
        assert tuple(t.shape) == self.shape, (tuple(t.shape), self.shape)
        return ct.c_void_p(t.data_ptr())

    def set_stream(self, stream) -> None:
        raw = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.lbm_unet_set_stream(self.h, ct.c_void_p(raw or 0)))

    @property
    def param_count(self) -> int:
        return int(self.lib.lbm_unet_param_count(self.h))

    @property
    def device_bytes(self) -> int:
        return int(self.lib.lbm_unet_device_bytes(self.h))

    def set_params(self, params) -> None:
        vec = flatten(params, self.shapes) if isinstance(params, dict) else np.asarray(params, np.float32)
        vec = np.ascontiguousarray(vec, np.float32)
        assert vec.size == self.param_count
        self._check(self.lib.lbm_unet_set_params(self.h, vec.ctypes.data_as(ct.c_void_p)))

    def _get(self, fn) -> dict:
        vec = np.empty(self.param_count, np.float32)
        self._check(fn(self.h, vec.ctypes.data_as(ct.c_void_p)))
        return unflatten(vec, self.shapes)

    def params(self) -> dict:
        return self._get(self.lib.lbm_unet_get_params)

    def grads(self) -> dict:
        return self._get(self.lib.lbm_unet_get_grads)

    def set_norm(self, mean, std) -> None:
        m = np.ascontiguousarray(mean, np.float32)
        s = np.ascontiguousarray(std, np.float32)
        assert m.size == self.fields and s.size == self.fields
        self._check(self.lib.lbm_unet_set_norm(self.h, m.ctypes.data_as(ct.c_void_p), s.ctypes.data_as(ct.c_void_p)))

    def forward(self, x, y=None):
        """Prediction in physical units (into `y` when given)."""
        import torch

        if y is None:
            y = torch.empty_like(x)
        self._check(self.lib.lbm_unet_forward(self.h, self._t(x), self._t(y)))
        return y

    def output_normalised(self):
        """The last prediction in normalised units (a new CUDA tensor)."""
        import torch

        out = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        self._check(self.lib.lbm_unet_output(self.h, self._t(out)))
        return out

    def backward(self, x, target) -> None:
        self._check(self.lib.lbm_unet_backward(self.h, self._t(x), self._t(target)))

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
        self._check(self.lib.lbm_unet_adam(self.h, lr, beta1, beta2, eps))

    def train_step(self, x, target, lr: float) -> None:
        self._check(self.lib.lbm_unet_train_step(self.h, self._t(x), self._t(target), lr))

    def loss(self) -> float:
        out = ct.c_double()
        self._check(self.lib.lbm_unet_loss(self.h, ct.byref(out)))
        return out.value
