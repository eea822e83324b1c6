"""Solutal dendrite of Sec. 4.3 on the GPU: the isothermal alloy (no latent
heat, reading R22) against the FP64 oracle, with and without melt flow."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2209_01444_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_2209_01444_gb300 import build_ext, lbm as L

    build_ext.build()
    L.load()
    return L


@pytest.mark.parametrize("flow", [False, True])
def test_isothermal_parity(lbm, flow):
    """64 x 64, 40 coupled steps (600 flow sub-steps with flow) of the Sec. 4.3
    parameter set against the oracle; theta stays exactly 0 on both sides."""
    from test_gpu_parity import FP32_TOL, field_errors

    n = 64
    p = W.solutal_params(n, flow=flow)
    seeds = np.array([[n / 2, n / 2, 6.0, 0.0]])
    g = lbm.Simulation(p)
    g.init_seeds(seeds, -0.55, 0.0)
    o = O.Oracle(p)
    o.init_seeds(seeds, -0.55, 0.0)
    g.step(40)
    o.step(40)
    fg, fo = g.fields(), o.fields()
    assert np.abs(fg["theta"]).max() == 0.0 and np.abs(fo["theta"]).max() == 0.0
    errs = field_errors(fg, fo, 0.55)
    print(f"isothermal parity (flow {flow}):", {k: f"{v:.2e}" for k, v in errs.items()})
    assert all(v <= FP32_TOL for v in errs.values()), errs
