"""ctypes binding of the C ABI in ``include/lbm.h`` (``liblbm.so``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The raw functions keep their C names (``lbm_create``,
``lbm_step``, ...); :class:`Simulation` wraps a handle for convenience.  There
is no CPU fallback: if ``liblbm.so`` cannot be loaded this module raises.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENUMERIC, LBM_ETIMEOUT, LBM_ESTATE = 0, -1, -2, -3, -4, -5, -6
BC = {"periodic": 0, "inflow": 1, "outflow": 2, "symmetry": 3, "noslip": 4, "dirichlet": 5}
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}
FIELDS = ("phi", "C", "U", "theta", "ux", "uy", "p")
STATE_PLANES = 30
ERRORS = {LBM_EINVAL: "EINVAL", LBM_ENOMEM: "ENOMEM", LBM_ECUDA: "ECUDA", LBM_ENUMERIC: "ENUMERIC",
          LBM_ETIMEOUT: "ETIMEOUT", LBM_ESTATE: "ESTATE"}


class lbm_params(ct.Structure):
    _fields_ = [
        ("nx", ct.c_int), ("ny", ct.c_int),
        ("W0", ct.c_double), ("tau0", ct.c_double), ("dx", ct.c_double), ("dt", ct.c_double),
        ("eps_s", ct.c_double), ("lambda_", ct.c_double), ("k", ct.c_double), ("Mc_inf", ct.c_double),
        ("D", ct.c_double), ("alpha", ct.c_double), ("nu", ct.c_double), ("rho0", ct.c_double),
        ("n_sub", ct.c_int), ("h_kind", ct.c_int),
        ("gbetaT", ct.c_double), ("gbetaC", ct.c_double), ("theta_ref", ct.c_double), ("C_ref", ct.c_double),
        ("force", ct.c_double * 2),
        ("bc", ct.c_int * 4),
        ("u_in", ct.c_double * 2),
        ("dir_phi", ct.c_double), ("dir_U", ct.c_double), ("dir_theta", ct.c_double),
        ("storage", ct.c_int),
        ("grad_mode", ct.c_int),
        ("isothermal", ct.c_int),
    ]


class lbm_seed(ct.Structure):
    _fields_ = [("x", ct.c_double), ("y", ct.c_double), ("R", ct.c_double), ("orient", ct.c_double)]


class lbm_surrogate_report(ct.Structure):
    _fields_ = [("audited", ct.c_int), ("accepted", ct.c_int), ("tip_err", ct.c_double),
                ("tip", ct.c_double * 3), ("mismatch", ct.c_longlong), ("max_dphi", ct.c_double)]


class lbm_metrics(ct.Structure):
    _fields_ = [("tip", ct.c_double * 3), ("solid_fraction", ct.c_double), ("sum_C", ct.c_double),
                ("sum_H", ct.c_double), ("sum_h", ct.c_double), ("max_u", ct.c_double),
                ("nonfinite", ct.c_double), ("sum_phi", ct.c_double), ("step", ct.c_longlong)]


# name -> (restype, argtypes) of every function declared in include/lbm.h
_H = ct.c_void_p
_DP = ct.POINTER(ct.c_double)
SIGNATURES = {
    "lbm_params_default": (ct.c_int, [ct.POINTER(lbm_params), ct.c_int, ct.c_int]),
    "lbm_create": (ct.c_int, [ct.POINTER(lbm_params), ct.POINTER(ct.c_void_p)]),
    "lbm_destroy": (None, [_H]),
    "lbm_set_stream": (ct.c_int, [_H, ct.c_void_p]),
    "lbm_init_seeds": (ct.c_int, [_H, ct.POINTER(lbm_seed), ct.c_int, ct.c_double, ct.c_double]),
    "lbm_init_fields": (ct.c_int, [_H, _DP, _DP]),
    "lbm_step": (ct.c_int, [_H, ct.c_int]),
    "lbm_set_io_chunk": (ct.c_int, [_H, ct.c_size_t]),
    "lbm_synchronize": (ct.c_int, [_H]),
    "lbm_step_count": (ct.c_longlong, [_H]),
    "lbm_get_fields": (ct.c_int, [_H, ct.c_uint, _DP]),
    "lbm_get_fields_f32": (ct.c_int, [_H, ct.c_uint, ct.c_void_p]),
    "lbm_get_state": (ct.c_int, [_H, _DP]),
    "lbm_get_state_region": (ct.c_int, [_H, ct.c_int, ct.c_int, ct.c_int, ct.c_int, _DP]),
    "lbm_set_state": (ct.c_int, [_H, _DP]),
    "lbm_get_metrics": (ct.c_int, [_H, ct.c_double, ct.c_double, ct.c_double, ct.POINTER(lbm_metrics)]),
    "lbm_checkpoint_bytes": (ct.c_size_t, [_H]),
    "lbm_save_state": (ct.c_int, [_H, ct.c_void_p, ct.c_size_t]),
    "lbm_load_state": (ct.c_int, [_H, ct.c_void_p, ct.c_size_t]),
    "lbm_reduce_noalloc": (ct.c_int, [ct.POINTER(lbm_params), ct.c_void_p, ct.c_void_p, ct.c_double, ct.c_double,
                                      ct.c_double, ct.c_void_p, ct.c_void_p]),
    "lbm_batch_create": (ct.c_int, [ct.POINTER(lbm_params), ct.c_int, ct.POINTER(ct.c_void_p)]),
    "lbm_batch_destroy": (None, [_H]),
    "lbm_batch_set_stream": (ct.c_int, [_H, ct.c_void_p]),
    "lbm_batch_init_seeds": (ct.c_int, [_H, ct.c_int, ct.POINTER(lbm_seed), ct.c_int, ct.c_double, ct.c_double]),
    "lbm_batch_step": (ct.c_int, [_H, ct.c_int]),
    "lbm_batch_synchronize": (ct.c_int, [_H]),
    "lbm_batch_get_fields": (ct.c_int, [_H, ct.c_int, ct.c_uint, _DP]),
    "lbm_batch_get_metrics": (ct.c_int, [_H, ct.c_int, ct.c_double, ct.c_double, ct.c_double,
                                         ct.POINTER(lbm_metrics)]),
    "lbm_batch_nodes": (ct.c_longlong, [_H]),
    "lbm_batch_tile_height": (ct.c_int, [_H]),
    "lbm_batch_tiles_per_cta": (ct.c_int, [_H]),
    "lbm_batch_set_tiling": (ct.c_int, [_H, ct.c_int, ct.c_int]),
    "lbm_batch_tune": (ct.c_int, [_H, ct.c_char_p, ct.POINTER(ct.c_int)]),
    "lbm_batch_set_profiling": (ct.c_int, [_H, ct.c_int]),
    "lbm_batch_kernel_time": (ct.c_int, [_H, ct.POINTER(ct.c_double), ct.POINTER(ct.c_longlong)]),
    "lbm_batch_last_error": (ct.c_char_p, [_H]),
    "lbm_nn_gemm": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p,
                               ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p]),
    "lbm_nn_error": (ct.c_int, [ct.c_int]),
    "lbm_nn_set_operand_wait": (ct.c_int, [ct.c_ulonglong]),
    "lbm_nn_gemm_split": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int,
                                     ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int,
                                     ct.c_void_p, ct.c_void_p]),
    "lbm_nn_im2col3x3": (ct.c_int, [ct.c_void_p] + [ct.c_int] * 5 + [ct.c_void_p, ct.c_void_p]),
    "lbm_nn_col2im3x3": (ct.c_int, [ct.c_void_p] + [ct.c_int] * 4 + [ct.c_void_p, ct.c_int, ct.c_void_p]),
    "lbm_nn_relu_bwd": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_int, ct.c_longlong, ct.c_int,
                                   ct.c_void_p]),
    "lbm_nn_transpose": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p]),
    "lbm_nn_maxpool_fwd": (ct.c_int, [ct.c_void_p] + [ct.c_int] * 5 + [ct.c_void_p, ct.c_void_p]),
    "lbm_nn_maxpool_bwd": (ct.c_int, [ct.c_void_p] + [ct.c_int] * 5 + [ct.c_void_p, ct.c_void_p, ct.c_int,
                                                                       ct.c_void_p]),
    "lbm_nn_shuffle_fwd": (ct.c_int, [ct.c_void_p] + [ct.c_int] * 4 + [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p]),
    "lbm_nn_shuffle_bwd": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int] + [ct.c_int] * 4 +
                           [ct.c_void_p, ct.c_void_p]),
    "lbm_nn_proj_fwd": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_int,
                                   ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "lbm_nn_proj_bwd": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p, ct.c_int,
                                   ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int,
                                   ct.c_void_p]),
    "lbm_nn_flip3x3": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p]),
    "lbm_nn_gather_t": (ct.c_int, [ct.c_void_p] + [ct.c_int] * 6 + [ct.c_void_p, ct.c_longlong, ct.c_void_p]),
    "lbm_nn_wgrad3x3": (ct.c_int, [ct.c_void_p, ct.c_void_p] + [ct.c_int] * 5 + [ct.c_void_p, ct.c_int, ct.c_int,
                                                                                ct.c_void_p, ct.c_void_p]),
    "lbm_nn_conv3x3": (ct.c_int, [ct.c_void_p] + [ct.c_int] * 5 + [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int,
                                                                    ct.c_void_p, ct.c_int, ct.c_int, ct.c_int,
                                                                    ct.c_void_p]),
    "lbm_nn_upconv2x2": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_void_p, ct.c_int, ct.c_int,
                                    ct.c_void_p] + [ct.c_int] * 5 + [ct.c_void_p]),
    "lbm_unet_create": (ct.c_int, [ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_void_p]),
    "lbm_unet_destroy": (None, [ct.c_void_p]),
    "lbm_unet_set_stream": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "lbm_unet_param_count": (ct.c_longlong, [ct.c_void_p]),
    "lbm_unet_device_bytes": (ct.c_longlong, [ct.c_void_p]),
    "lbm_unet_set_params": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "lbm_unet_get_params": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "lbm_unet_get_grads": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "lbm_unet_set_norm": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "lbm_unet_set_loss_weight": (ct.c_int, [ct.c_void_p, ct.c_float]),
    "lbm_unet_save": (ct.c_int, [ct.c_void_p, ct.c_char_p]),
    "lbm_unet_load": (ct.c_int, [ct.c_void_p, ct.c_char_p]),
    "lbm_unet_forward": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "lbm_unet_backward": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    "lbm_unet_adam": (ct.c_int, [ct.c_void_p, ct.c_float, ct.c_float, ct.c_float, ct.c_float]),
    "lbm_unet_train_step": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_float]),
    "lbm_unet_loss": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "lbm_unet_output": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "lbm_unet_last_error": (ct.c_char_p, [ct.c_void_p]),
    "lbm_unet_shape": (ct.c_int, [ct.c_void_p] + [ct.POINTER(ct.c_int)] * 4),
    "lbm_step_flow": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "lbm_get_force": (ct.c_int, [ct.c_void_p, ct.c_double, ct.c_double, ct.c_void_p]),
    "lbm_set_monitor": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_int, ct.c_double, ct.c_double, ct.c_double]),
    "lbm_get_monitor": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int, ct.POINTER(ct.c_int)]),
    "lbm_snapshot_save": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "lbm_snapshot_restore": (ct.c_int, [ct.c_void_p, ct.c_int]),
    "lbm_fields_nhwc": (ct.c_int, [ct.c_void_p, ct.c_void_p]),
    "lbm_set_fields_nhwc": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int]),
    "lbm_batch_fields_nhwc": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_void_p]),
    "lbm_surrogate_advance": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int, ct.c_double, ct.c_int, ct.c_double,
                                         ct.c_double, ct.c_double, ct.c_void_p]),
    "lbm_nn_colsum": (ct.c_int, [ct.c_void_p, ct.c_int, ct.c_longlong, ct.c_int, ct.c_int, ct.c_void_p, ct.c_void_p,
                                 ct.c_int, ct.c_void_p]),
    "lbm_nn_mse": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_longlong, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                              ct.c_void_p]),
    "lbm_nn_adam": (ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_longlong, ct.c_float,
                               ct.c_float, ct.c_float, ct.c_float, ct.c_int, ct.c_void_p, ct.c_void_p]),
    "lbm_nn_pack": (ct.c_int, [ct.c_void_p, ct.c_longlong, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int,
                               ct.c_void_p, ct.c_void_p]),
    "lbm_nn_unpack": (ct.c_int, [ct.c_void_p, ct.c_longlong, ct.c_int, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                 ct.c_void_p]),
    "lbm_nn_cast_bf16": (ct.c_int, [ct.c_void_p, ct.c_longlong, ct.c_int, ct.c_int, ct.c_void_p, ct.c_int,
                                    ct.c_void_p]),

    "lbm_set_profiling": (ct.c_int, [_H, ct.c_int]),
    "lbm_kernel_time": (ct.c_int, [_H, _DP, ct.POINTER(ct.c_longlong)]),
    "lbm_last_error": (ct.c_char_p, [_H]),
    "lbm_version": (ct.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load ``liblbm.so`` and declare every C-ABI function; raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the library has no CPU fallback)")
    lib = ct.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def make_params(p: dict, storage: str | int = "fp32") -> lbm_params:
    """Fill an ``lbm_params`` from a problem dict (keys as in the paper's
    statement, see ``workloads``)."""
    s = lbm_params()
    for name, _ in lbm_params._fields_:
        if name == "storage":
            s.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
            continue
        v = p[name]
        if name == "bc":
            for i, b in enumerate(v):
                s.bc[i] = BC[b] if isinstance(b, str) else int(b)
        elif name in ("force", "u_in"):
            arr = getattr(s, name)
            arr[0], arr[1] = float(v[0]), float(v[1])
        else:
            setattr(s, name, v)
    return s


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


class Simulation:
    """One domain on the current CUDA device."""

    def __init__(self, params: dict, storage: str | int = "fp32", stream=None):
        self.lib = load()
        self.params = dict(params)
        self._p = make_params(params, storage)
        h = ct.c_void_p()
        rc = self.lib.lbm_create(ct.byref(self._p), ct.byref(h))
        if rc != LBM_OK:
            raise LBMError(rc, self.lib.lbm_last_error(None).decode())
        self.h = h
        self.nx, self.ny = int(params["nx"]), int(params["ny"])
        if stream is not None:
            self.set_stream(stream)

    def _check(self, rc: int) -> None:
        if rc != LBM_OK:
            raise LBMError(rc, self.lib.lbm_last_error(self.h).decode())

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h:
            self.lib.lbm_destroy(h)

    def set_stream(self, stream) -> None:
        """Accepts a ``torch.cuda.Stream``, a raw ``cudaStream_t`` int, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.lbm_set_stream(self.h, ct.c_void_p(raw or 0)))

    def init_seeds(self, seeds, U0: float, theta0: float) -> None:
        a = np.asarray(seeds, np.float64).reshape(-1, 4)
        arr = (lbm_seed * len(a))(*[lbm_seed(*row) for row in a])
        self._check(self.lib.lbm_init_seeds(self.h, arr, len(a), U0, theta0))

    def init_fields(self, fields: np.ndarray, orient: np.ndarray | None = None) -> None:
        f = np.ascontiguousarray(np.asarray(fields, np.float64).reshape(6, self.ny, self.nx))
        o = None if orient is None else np.ascontiguousarray(np.asarray(orient, np.float64).reshape(self.ny, self.nx))
        self._check(self.lib.lbm_init_fields(self.h, _dptr(f), None if o is None else _dptr(o)))

    def step(self, n: int = 1) -> None:
        self._check(self.lib.lbm_step(self.h, int(n)))

    def synchronize(self) -> None:
        self._check(self.lib.lbm_synchronize(self.h))

    def set_io_chunk(self, nbytes: int) -> None:
        """Size limit of the device band buffer of whole-grid transfers."""
        self._check(self.lib.lbm_set_io_chunk(self.h, int(nbytes)))

    @property
    def steps(self) -> int:
        return int(self.lib.lbm_step_count(self.h))

    def fields(self, names=FIELDS) -> dict:
        mask = 0
        for n in names:
            mask |= 1 << FIELDS.index(n)
        order = [n for n in FIELDS if mask & (1 << FIELDS.index(n))]
        out = np.empty((len(order), self.ny, self.nx))
        self._check(self.lib.lbm_get_fields(self.h, mask, _dptr(out)))
        return {n: out[i] for i, n in enumerate(order)}

    def fields_f32(self, names=FIELDS, out=None) -> dict:
        """FP32 fields through lbm_get_fields_f32; `out` (float32, C order,
        [len(names), ny, nx]) may be page-locked memory the caller keeps."""
        mask = 0
        for n in names:
            mask |= 1 << FIELDS.index(n)
        order = [n for n in FIELDS if mask & (1 << FIELDS.index(n))]
        if out is None:
            out = np.empty((len(order), self.ny, self.nx), np.float32)
        assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == len(order) * self.ny * self.nx
        out = out.reshape(len(order), self.ny, self.nx)
        self._check(self.lib.lbm_get_fields_f32(self.h, mask, ct.c_void_p(out.ctypes.data)))
        return {n: out[i] for i, n in enumerate(order)}

    def state(self) -> np.ndarray:
        out = np.empty((STATE_PLANES, self.ny, self.nx))
        self._check(self.lib.lbm_get_state(self.h, _dptr(out)))
        return out

    def state_region(self, x0: int, y0: int, w: int, hgt: int) -> np.ndarray:
        out = np.empty((STATE_PLANES, hgt, w))
        self._check(self.lib.lbm_get_state_region(self.h, x0, y0, w, hgt, _dptr(out)))
        return out

    def set_state(self, st: np.ndarray) -> None:
        a = np.ascontiguousarray(np.asarray(st, np.float64).reshape(STATE_PLANES, self.ny, self.nx))
        self._check(self.lib.lbm_set_state(self.h, _dptr(a)))

    def metrics(self, cx: float, cy: float, orient: float = 0.0, check: bool = True) -> dict:
        m = lbm_metrics()
        rc = self.lib.lbm_get_metrics(self.h, cx, cy, orient, ct.byref(m))
        if check:
            self._check(rc)
        return {"tip_px": m.tip[0], "tip_mx": m.tip[1], "tip_py": m.tip[2], "solid_fraction": m.solid_fraction,
                "sum_C": m.sum_C, "sum_H": m.sum_H, "sum_h": m.sum_h, "max_u": m.max_u,
                "nonfinite": m.nonfinite, "sum_phi": m.sum_phi, "step": m.step, "rc": rc}

    # ---- flow-only steps and the hydrodynamic force
    def step_flow(self, n: int = 1) -> None:
        """n steps of the flow model alone, phi, C and theta frozen."""
        self._check(self.lib.lbm_step_flow(self.h, int(n)))

    def force(self, cx: float, cy: float) -> tuple[float, float, float]:
        """Hydrodynamic force (x, y) on the solid and torque about (cx, cy), flow lattice units."""
        out = np.empty(3)
        self._check(self.lib.lbm_get_force(self.h, cx, cy, out.ctypes.data_as(ct.c_void_p)))
        return float(out[0]), float(out[1]), float(out[2])

    # ---- periodic reductions
    def set_monitor(self, every: int, capacity: int, cx: float, cy: float, orient: float = 0.0) -> None:
        self._check(self.lib.lbm_set_monitor(self.h, int(every), int(capacity), cx, cy, orient))

    def monitor(self, max_records: int = 1 << 20) -> list[dict]:
        """Recorded metrics, oldest first, each with the tip velocities v_tip
        (paper units; NaN for the first record)."""
        cap = max(1, int(max_records))
        arr = (lbm_metrics * cap)()
        v = np.empty(3 * cap)
        n = ct.c_int()
        self._check(self.lib.lbm_get_monitor(self.h, arr, v.ctypes.data_as(ct.c_void_p), cap, ct.byref(n)))
        out = []
        for i in range(n.value):
            m = arr[i]
            out.append({"step": m.step, "tip_px": m.tip[0], "tip_mx": m.tip[1], "tip_py": m.tip[2],
                        "v_px": v[3 * i], "v_mx": v[3 * i + 1], "v_py": v[3 * i + 2],
                        "solid_fraction": m.solid_fraction, "sum_C": m.sum_C, "sum_H": m.sum_H, "sum_h": m.sum_h,
                        "max_u": m.max_u, "nonfinite": m.nonfinite, "sum_phi": m.sum_phi})
        return out

    # ---- device-side exchange with the surrogate network
    def snapshot_save(self, slot: int = 0) -> None:
        self._check(self.lib.lbm_snapshot_save(self.h, slot))

    def snapshot_restore(self, slot: int = 0) -> None:
        self._check(self.lib.lbm_snapshot_restore(self.h, slot))

    def fields_nhwc(self, out=None):
        """Device FP32 tensor [ny, nx, 5] of phi, C, theta, u_x, u_y."""
        import torch

        if out is None:
            out = torch.empty(self.ny, self.nx, 5, dtype=torch.float32, device="cuda")
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.numel() == self.ny * self.nx * 5
        self._check(self.lib.lbm_fields_nhwc(self.h, ct.c_void_p(out.data_ptr())))
        return out

    def set_fields_nhwc(self, src, prev=None, K: int = 0) -> None:
        import torch

        for t in (src,) if prev is None else (src, prev):
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == self.ny * self.nx * 5
        self._check(self.lib.lbm_set_fields_nhwc(self.h, ct.c_void_p(src.data_ptr()),
                                                 None if prev is None else ct.c_void_p(prev.data_ptr()), int(K)))

    def surrogate_advance(self, net, K: int, tip_tol: float, audit: bool, cx: float, cy: float,
                          orient: float = 0.0) -> dict:
        rep = lbm_surrogate_report()
        self._check(self.lib.lbm_surrogate_advance(self.h, net.h, K, tip_tol, 1 if audit else 0, cx, cy, orient,
                                                   ct.byref(rep)))
        return {"audited": bool(rep.audited), "accepted": bool(rep.accepted), "tip_err": rep.tip_err,
                "tip": tuple(rep.tip), "mismatch": rep.mismatch, "max_dphi": rep.max_dphi}

    def set_profiling(self, enable: bool, what: str = "fused") -> None:
        """Time the fused kernel (`what` = "fused") or the flow sub-step
        kernels ("substep") of every coupled step with CUDA events."""
        mode = 0 if not enable else {"fused": 1, "substep": 2}[what]
        self._check(self.lib.lbm_set_profiling(self.h, mode))

    def kernel_time(self) -> tuple[float, int]:
        """(total ms, launches) of the timed kernels since profiling was enabled."""
        ms, n = ct.c_double(), ct.c_longlong()
        self._check(self.lib.lbm_kernel_time(self.h, ct.byref(ms), ct.byref(n)))
        return ms.value, n.value

    def save(self) -> bytes:
        n = self.lib.lbm_checkpoint_bytes(self.h)
        buf = ct.create_string_buffer(n)
        self._check(self.lib.lbm_save_state(self.h, buf, n))
        return buf.raw

    def load(self, blob: bytes) -> None:
        buf = ct.create_string_buffer(blob, len(blob))
        self._check(self.lib.lbm_load_state(self.h, buf, len(blob)))


class Batch:
    """Independent domains advanced together by the batched persistent kernel."""

    def __init__(self, params_list, storage: str | int = "fp32", stream=None):
        self.lib = load()
        self.params = [dict(p) for p in params_list]
        arr = (lbm_params * len(params_list))(*[make_params(p, storage) for p in params_list])
        h = ct.c_void_p()
        rc = self.lib.lbm_batch_create(arr, len(params_list), ct.byref(h))
        if rc != LBM_OK:
            raise LBMError(rc, self.lib.lbm_batch_last_error(None).decode())
        self.h = h
        if stream is not None:
            raw = getattr(stream, "cuda_stream", stream)
            self._check(self.lib.lbm_batch_set_stream(self.h, ct.c_void_p(raw or 0)))

    def _check(self, rc: int) -> None:
        if rc != LBM_OK:
            raise LBMError(rc, self.lib.lbm_batch_last_error(self.h).decode())

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h:
            self.lib.lbm_batch_destroy(h)

    def __len__(self):
        return len(self.params)

    @property
    def nodes(self) -> int:
        return int(self.lib.lbm_batch_nodes(self.h))

    @property
    def tile_height(self) -> int:
        return int(self.lib.lbm_batch_tile_height(self.h))

    @property
    def tiles_per_cta(self) -> int:
        return int(self.lib.lbm_batch_tiles_per_cta(self.h))

    def set_tiling(self, tile_height: int, tiles_per_cta: int = 1) -> None:
        self._check(self.lib.lbm_batch_set_tiling(self.h, int(tile_height), int(tiles_per_cta)))

    def init_seeds(self, dom: int, seeds, U0: float, theta0: float) -> None:
        a = np.asarray(seeds, np.float64).reshape(-1, 4)
        arr = (lbm_seed * len(a))(*[lbm_seed(*row) for row in a])
        self._check(self.lib.lbm_batch_init_seeds(self.h, dom, arr, len(a), U0, theta0))

    def set_profiling(self, enable: bool) -> None:
        """Time the batched kernel of every step with CUDA events (direct launches)."""
        self._check(self.lib.lbm_batch_set_profiling(self.h, int(enable)))

    def kernel_time(self) -> tuple[float, int]:
        """(total ms, launches) of the batched kernel since profiling was enabled."""
        ms, n = ct.c_double(), ct.c_longlong()
        self._check(self.lib.lbm_batch_kernel_time(self.h, ct.byref(ms), ct.byref(n)))
        return ms.value, n.value

    def tune(self, cache_path: str | None = None) -> int:
        ty = ct.c_int()
        self._check(self.lib.lbm_batch_tune(self.h, cache_path.encode() if cache_path else None, ct.byref(ty)))
        return ty.value

    def step(self, n: int = 1) -> None:
        self._check(self.lib.lbm_batch_step(self.h, int(n)))

    def synchronize(self) -> None:
        self._check(self.lib.lbm_batch_synchronize(self.h))

    def fields(self, dom: int, names=FIELDS) -> dict:
        nx, ny = int(self.params[dom]["nx"]), int(self.params[dom]["ny"])
        mask = 0
        for n in names:
            mask |= 1 << FIELDS.index(n)
        order = [n for n in FIELDS if mask & (1 << FIELDS.index(n))]
        out = np.empty((len(order), ny, nx))
        self._check(self.lib.lbm_batch_get_fields(self.h, dom, mask, _dptr(out)))
        return {n: out[i] for i, n in enumerate(order)}

    def fields_nhwc(self, dom: int, out):
        """Writes domain `dom`'s phi, C, theta, u_x, u_y into the device FP32
        tensor `out` [ny, nx, 5]."""
        import torch

        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
        p = self.params[dom]
        assert out.numel() == int(p["nx"]) * int(p["ny"]) * 5
        self._check(self.lib.lbm_batch_fields_nhwc(self.h, dom, ct.c_void_p(out.data_ptr())))
        return out

    def metrics(self, dom: int, cx: float, cy: float, orient: float = 0.0) -> dict:
        m = lbm_metrics()
        self._check(self.lib.lbm_batch_get_metrics(self.h, dom, cx, cy, orient, ct.byref(m)))
        return {"tip_px": m.tip[0], "tip_mx": m.tip[1], "tip_py": m.tip[2], "solid_fraction": m.solid_fraction,
                "sum_C": m.sum_C, "sum_H": m.sum_H, "sum_h": m.sum_h, "max_u": m.max_u,
                "nonfinite": m.nonfinite, "sum_phi": m.sum_phi, "step": m.step}
