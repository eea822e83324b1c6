"""ctypes binding of the FP64 CPU oracle in ``lbm_oracle.c``.

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow FP64 statement of the
diffuse-interface MRT lattice Boltzmann method of arXiv 2209.01444 that the CUDA
path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
module.  It never imports the CUDA package, and the CUDA package never
imports it.

Parameters are plain dicts whose keys are the fields of ``orc_params``
(``nx, ny, W0, tau0, dx, dt, eps_s, lambda_, k, Mc_inf, D, alpha, nu, rho0,
n_sub, h_kind, gbetaT, gbetaC, theta_ref, C_ref, force, bc, u_in, dir_phi,
dir_U, dir_theta``); ``lambda_`` stands for the paper's coupling constant.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

FIELDS = ("phi", "C", "U", "theta", "ux", "uy", "p")
BC = {"periodic": 0, "inflow": 1, "outflow": 2, "symmetry": 3, "noslip": 4, "dirichlet": 5}


class _Params(ct.Structure):
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
        ("grad_mode", ct.c_int),
        ("isothermal", ct.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` into ``liblbm_oracle.so`` beside it (portable
    flags only: the same source builds on x86-64 and aarch64)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                      os.path.getmtime(os.path.join(_HERE, "lbm_oracle.h")))):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ct.CDLL(_LIB_PATH)
    dp = ct.POINTER(ct.c_double)
    lib.orc_create.restype = ct.c_void_p
    lib.orc_create.argtypes = [ct.POINTER(_Params)]
    lib.orc_destroy.argtypes = [ct.c_void_p]
    lib.orc_init_seeds.argtypes = [ct.c_void_p, dp, ct.c_int, ct.c_double, ct.c_double]
    lib.orc_init_seeds_window.argtypes = [ct.c_void_p, dp, ct.c_int, ct.c_double, ct.c_double] + [ct.c_int] * 6
    lib.orc_init_fields.argtypes = [ct.c_void_p, dp, dp]
    lib.orc_step.argtypes = [ct.c_void_p, ct.c_int]
    lib.orc_step_flow.argtypes = [ct.c_void_p, ct.c_int]
    lib.orc_force.argtypes = [ct.c_void_p, ct.c_double, ct.c_double, dp]
    lib.orc_grad_phi.argtypes = [ct.c_void_p, ct.c_int, dp]
    lib.orc_step_count.restype = ct.c_longlong
    lib.orc_step_count.argtypes = [ct.c_void_p]
    for name in ("orc_get_fields", "orc_get_state", "orc_set_state", "orc_get_orient", "orc_lattice_params"):
        getattr(lib, name).argtypes = [ct.c_void_p, dp]
    lib.orc_metrics.argtypes = [ct.c_void_p, ct.c_double, ct.c_double, ct.c_double, dp]
    lib.orc_lattice_M5.argtypes = [dp]
    lib.orc_lattice_M9.argtypes = [dp]
    lib.orc_lambda5.argtypes = [ct.c_double, ct.c_double, ct.c_double, dp]
    lib.orc_lambda9.argtypes = [dp, dp]
    lib.orc_feq_phi.argtypes = [ct.c_double, dp]
    lib.orc_F_phi.argtypes = [ct.c_double, ct.c_double, dp]
    lib.orc_G_phi.argtypes = [ct.c_double, ct.c_double, ct.c_double, dp]
    lib.orc_neq.argtypes = [ct.c_double] * 4 + [dp]
    lib.orc_G_C.argtypes = [ct.c_double] * 8 + [dp]
    lib.orc_geq.argtypes = [ct.c_double] * 4 + [dp]
    lib.orc_G_theta.argtypes = [ct.c_double] * 2 + [dp]
    lib.orc_heq.argtypes = [ct.c_double] * 4 + [dp]
    lib.orc_F_u.argtypes = [ct.c_double] * 2 + [dp]
    lib.orc_anisotropy.argtypes = [ct.c_double] * 4 + [dp, dp, dp]
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _to_struct(p: dict) -> _Params:
    s = _Params()
    for name, typ in _Params._fields_:
        if name not in p:
            raise KeyError(f"missing parameter {name!r}")
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


class Oracle:
    """One FP64 simulation.  Fields are returned as (ny, nx) arrays."""

    def __init__(self, params: dict):
        self.lib = _load()
        self.params = dict(params)
        self._st = _to_struct(params)
        self.h = self.lib.orc_create(ct.byref(self._st))
        if not self.h:
            raise ValueError("oracle rejected the parameters")
        self.nx, self.ny = int(params["nx"]), int(params["ny"])

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h:
            self.lib.orc_destroy(h)

    @property
    def n(self) -> int:
        return self.nx * self.ny

    def init_seeds(self, seeds, U0: float, theta0: float) -> None:
        a = np.ascontiguousarray(np.asarray(seeds, dtype=np.float64).reshape(-1, 4))
        if self.lib.orc_init_seeds(self.h, _ptr(a), a.shape[0], U0, theta0):
            raise ValueError("init_seeds failed")

    def init_seeds_window(self, seeds, U0: float, theta0: float, x0: int, y0: int, gnx: int, gny: int,
                          periodic_x: bool, periodic_y: bool) -> None:
        """Seeded start of the window with lower-left node (x0, y0) of a larger
        gnx x gny domain (seed coordinates in that domain)."""
        a = np.ascontiguousarray(np.asarray(seeds, dtype=np.float64).reshape(-1, 4))
        if self.lib.orc_init_seeds_window(self.h, _ptr(a), a.shape[0], U0, theta0, x0, y0, gnx, gny,
                                          int(periodic_x), int(periodic_y)):
            raise ValueError("init_seeds_window failed")

    def init_fields(self, fields: np.ndarray, orient: np.ndarray | None = None) -> None:
        f = np.ascontiguousarray(np.asarray(fields, dtype=np.float64).reshape(6, self.n))
        o = None if orient is None else np.ascontiguousarray(np.asarray(orient, np.float64).reshape(self.n))
        if self.lib.orc_init_fields(self.h, _ptr(f), None if o is None else _ptr(o)):
            raise ValueError("init_fields failed")

    def step(self, n: int = 1) -> None:
        if self.lib.orc_step(self.h, int(n)):
            raise ValueError("step failed")

    def step_flow(self, n: int = 1) -> None:
        """n flow-only steps with phi, C, theta frozen."""
        if self.lib.orc_step_flow(self.h, int(n)):
            raise ValueError("step_flow failed")

    def force(self, cx: float, cy: float) -> tuple[float, float, float]:
        """Hydrodynamic force (x, y) and torque about (cx, cy), flow lattice units."""
        out = np.empty(3)
        self.lib.orc_force(self.h, cx, cy, _ptr(out))
        return float(out[0]), float(out[1]), float(out[2])

    def grad_phi(self, mode: int) -> np.ndarray:
        """grad(phi) [2, ny, nx] (lattice units) by the stencil (0) or the
        local scheme (1) from the current state."""
        out = np.empty((2, self.ny, self.nx))
        if self.lib.orc_grad_phi(self.h, int(mode), _ptr(out)):
            raise ValueError("grad_phi failed")
        return out

    @property
    def steps(self) -> int:
        return int(self.lib.orc_step_count(self.h))

    def fields(self) -> dict:
        out = np.empty((7, self.ny, self.nx))
        self.lib.orc_get_fields(self.h, _ptr(out))
        return {k: out[i] for i, k in enumerate(FIELDS)}

    def state(self) -> np.ndarray:
        out = np.empty((30, self.ny, self.nx))
        self.lib.orc_get_state(self.h, _ptr(out))
        return out

    def set_state(self, st: np.ndarray) -> None:
        a = np.ascontiguousarray(np.asarray(st, np.float64).reshape(30, self.ny, self.nx))
        self.lib.orc_set_state(self.h, _ptr(a))

    def orient(self) -> np.ndarray:
        out = np.empty((self.ny, self.nx))
        self.lib.orc_get_orient(self.h, _ptr(out))
        return out

    def metrics(self, cx: float, cy: float, orient: float = 0.0) -> dict:
        out = np.empty(10)
        self.lib.orc_metrics(self.h, cx, cy, orient, _ptr(out))
        keys = ("tip_px", "tip_mx", "tip_py", "solid_fraction", "sum_C", "sum_H", "sum_h",
                "max_u", "nonfinite", "sum_phi")
        return dict(zip(keys, out.tolist()))

    def lattice_params(self) -> dict:
        out = np.empty(9)
        self.lib.orc_lattice_params(self.h, _ptr(out))
        keys = ("W", "tau", "kappa0", "D", "s1C", "s1T", "s2u", "vscale", "fscale")
        return dict(zip(keys, out.tolist()))


# ------------------------------------------------------------ building blocks
def _vec(n, fn, *args):
    out = np.empty(n)
    fn(*args, _ptr(out))
    return out


def lattice_M5() -> np.ndarray:
    return _vec(25, _load().orc_lattice_M5).reshape(5, 5)


def lattice_M9() -> np.ndarray:
    return _vec(81, _load().orc_lattice_M9).reshape(9, 9)


def lambda5(s0, s1, s2) -> np.ndarray:
    return _vec(25, _load().orc_lambda5, s0, s1, s2).reshape(5, 5)


def lambda9(S) -> np.ndarray:
    S = np.ascontiguousarray(np.asarray(S, np.float64))
    return _vec(81, _load().orc_lambda9, _ptr(S)).reshape(9, 9)


def feq_phi(phi):
    return _vec(5, _load().orc_feq_phi, phi)


def F_phi(Q, tau):
    return _vec(5, _load().orc_F_phi, Q, tau)


def G_phi(Nx, Ny, as2):
    return _vec(5, _load().orc_G_phi, Nx, Ny, as2)


def neq(C, qU, Cux, Cuy):
    return _vec(5, _load().orc_neq, C, qU, Cux, Cuy)


def G_C(dCux, dCuy, U, gqx, gqy, Jx, Jy, D):
    return _vec(5, _load().orc_G_C, dCux, dCuy, U, gqx, gqy, Jx, Jy, D)


def geq(theta, Lh, Hux, Huy):
    return _vec(5, _load().orc_geq, theta, Lh, Hux, Huy)


def G_theta(dHux, dHuy):
    return _vec(5, _load().orc_G_theta, dHux, dHuy)


def heq(p, ux, uy, rho0):
    return _vec(9, _load().orc_heq, p, ux, uy, rho0)


def F_u(Fx, Fy):
    return _vec(9, _load().orc_F_u, Fx, Fy)


def anisotropy(gx, gy, eps, orient=0.0):
    a, nx_, ny_ = ct.c_double(), ct.c_double(), ct.c_double()
    _load().orc_anisotropy(gx, gy, eps, orient, ct.byref(a), ct.byref(nx_), ct.byref(ny_))
    return a.value, nx_.value, ny_.value
