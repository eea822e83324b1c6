"""Full-size parity on sampled windows.

The bench workloads are too large for the oracle to step whole, so the GPU runs
them at full size (same kernels, same launch configuration) for K coupled
steps from the seeded start, and the oracle computes windows of the same
problem from its own seeded start of that window (seed positions in the
coordinates of the full grid).  A node's state after K steps depends only on
nodes within 2K of it (one node of streaming plus one node of the phi stencil
per step), so the centre of a window with a margin larger than 2K is exact;
the comparison covers the centre only.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O
from paper_2209_01444_gb300 import workloads as W

pytestmark = pytest.mark.gpu
K = 4
MARGIN = 2 * K + 2
TOL = 2e-5  # absolute, on populations and history of magnitude <= ~1


@pytest.fixture(scope="module")
def lbm():
    import torch

    from paper_2209_01444_gb300 import build_ext, lbm as L

    build_ext.build()
    L.load()
    torch.cuda.init()
    return L


def oracle_window(case, x0, y0, w, h, bc):
    """Oracle run of the window [x0, x0+w) x [y0, y0+h) of the case's grid."""
    p = dict(case.params)
    p["nx"], p["ny"], p["bc"] = w, h, bc
    o = O.Oracle(p)
    N, M = case.params["nx"], case.params["ny"]
    per_x = case.params["bc"][0] == "periodic"
    per_y = case.params["bc"][2] == "periodic"
    o.init_seeds_window(case.seeds, case.U0, case.theta0, x0 % N, y0 % M, N, M, per_x, per_y)
    o.step(K)
    return o.state()


# FP16 storage: a stored deviation |d| <= 1 is rounded to 11 bits after the
# scale of 16 (flow: 1024), at most 2^-11 / 2 per rounding; four steps of
# rounding and mixing stay within 2e-3.
TOL16 = 2e-3


def compare(g, case, cx, cy, size, bc, ylo_wall=False, xlo_wall=False, tol=TOL):
    """GPU state of the size x size block at (cx, cy) against the oracle's
    window around it (margin on every side that is not a real wall)."""
    x0 = cx - (0 if xlo_wall else MARGIN)
    y0 = cy - (0 if ylo_wall else MARGIN)
    w = size + MARGIN * (1 if xlo_wall else 2)
    h = size + MARGIN * (1 if ylo_wall else 2)
    ref = oracle_window(case, x0, y0, w, h, bc)
    ox, oy = cx - x0, cy - y0
    want = ref[:, oy:oy + size, ox:ox + size]
    got = g.state_region(cx, cy, size, size)
    err = np.abs(got - want).max(axis=(1, 2))
    assert err.max() < tol, f"window ({cx},{cy}): worst plane {int(err.argmax())} error {err.max():.2e}"
    return float(err.max())


def test_multi_seed_4096_windows(lbm):
    """The 4096^2, 64-seed bench workload (periodic x, no-slip y)."""
    case = W.multi_seed()
    g = lbm.Simulation(case.params)
    g.init_seeds(case.seeds, case.U0, case.theta0)
    g.step(K)
    per = ("periodic",) * 4
    for j in (0, 17, 40):
        sx, sy = int(case.seeds[j][0]), int(case.seeds[j][1])
        compare(g, case, sx - 16, sy - 16, 32, per)
    compare(g, case, 1000, 2000, 32, per)                       # liquid far from seeds
    compare(g, case, 3000, 0, 24, ("periodic", "periodic", "noslip", "noslip"), ylo_wall=True)


def test_forced_flow_1024_windows(lbm):
    """The 1024^2 single-dendrite forced-flow workload (inflow left, outflow
    right, symmetry top and bottom)."""
    case = W.forced_flow()
    g = lbm.Simulation(case.params)
    g.init_seeds(case.seeds, case.U0, case.theta0)
    g.step(K)
    per = ("periodic",) * 4
    compare(g, case, 384 - 16, 512 - 16, 32, per)              # around the seed
    compare(g, case, 0, 600, 24, ("inflow", "outflow", "periodic", "periodic"), xlo_wall=True)
    compare(g, case, 500, 0, 24, ("periodic", "periodic", "symmetry", "symmetry"), ylo_wall=True)


def test_multi_seed_4096_windows_fp16(lbm):
    """The same workload with FP16 population storage, as the bench's FP16
    line runs it."""
    case = W.multi_seed()
    g = lbm.Simulation(case.params, "fp16")
    g.init_seeds(case.seeds, case.U0, case.theta0)
    g.step(K)
    per = ("periodic",) * 4
    worst = 0.0
    for j in (0, 40):
        sx, sy = int(case.seeds[j][0]), int(case.seeds[j][1])
        worst = max(worst, compare(g, case, sx - 16, sy - 16, 32, per, tol=TOL16))
    worst = max(worst, compare(g, case, 3000, 0, 24, ("periodic", "periodic", "noslip", "noslip"), ylo_wall=True,
                               tol=TOL16))
    print(f"FP16 full-size windows: worst population error {worst:.2e}")
