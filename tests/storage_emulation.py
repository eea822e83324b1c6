"""Rounding of an oracle state as the equilibrium-shifted 16-bit population
storage rounds it (test helper; no GPU).

Each population is held as its deviation from the equilibrium of the liquid at
rest (phi = -1, C = 1, theta = theta_ref, p = 0, u = 0).  FP16 storage scales
the deviation (16 for the scalar models, 1024 for the flow), rounds it to FP16
(nearest even) and scales back; BF16 rounds the unscaled deviation to BF16
(nearest even).  The three scalar rest populations and the six history planes
stay FP32.  Applied to the FP64 oracle after every step, this separates what
16-bit storage does to a state from what the kernels do."""
from __future__ import annotations

import numpy as np

W5 = np.array([1 / 3, 1 / 6, 1 / 6, 1 / 6, 1 / 6])
REST = (0, 5, 10)


def reference(params: dict) -> np.ndarray:
    """Populations 0..23 of the reference state (phi, C, H, flow)."""
    ref = np.zeros(24)
    ref[0:5] = -W5
    ref[5] = 1.0
    ref[10:15] = W5 * params["theta_ref"]
    ref[10] += 0.5 * (1 - params.get("isothermal", 0))
    ref[15] = params["rho0"]
    return ref


def bf16_round(x: np.ndarray) -> np.ndarray:
    """FP32 values rounded to BF16 (nearest, ties to even), as FP32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def round_state(o, params: dict, storage: str) -> None:
    """Round the oracle `o`'s state in place as `storage` ('fp16' or 'bf16') stores it."""
    ref = reference(params)
    st = o.state()
    for q in range(24):
        dev = (st[q] - ref[q]).astype(np.float32)
        if q in REST:
            st[q] = ref[q] + dev.astype(np.float64)
        elif storage == "fp16":
            sc = np.float32(1024.0 if q >= 15 else 16.0)
            st[q] = ref[q] + (np.float16(dev * sc).astype(np.float32) / sc).astype(np.float64)
        else:
            st[q] = ref[q] + bf16_round(dev).astype(np.float64)
    st[24:] = st[24:].astype(np.float32).astype(np.float64)
    o.set_state(st)
