"""Flow past a stationary cylinder (Sec. 4.1): flow-only steps and the
hydrodynamic force on the GPU against the oracle, and the drag coefficient
and recirculation length of the full-size case against Table 1."""
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


def test_flow_steps_and_force_match_oracle(lbm):
    c = W.cylinder_flow(Re=20.0, nx=120, ny=80, R=8.0)
    c.seeds[0, :2] = (40.0, 40.0)
    sim = lbm.Simulation(c.params)
    sim.init_seeds(c.seeds, c.U0, c.theta0)
    o = O.Oracle(c.params)
    o.init_seeds(c.seeds, c.U0, c.theta0)
    sim.step_flow(300)
    o.step_flow(300)
    g, r = sim.fields(("ux", "uy", "p", "phi")), o.fields()
    umax = np.abs(r["ux"]).max()
    for k in ("ux", "uy"):
        assert np.abs(g[k] - r[k]).max() <= 1e-4 * umax, k
    assert np.abs(g["p"] - r["p"]).max() <= 1e-4 * max(np.abs(r["p"]).max(), 1e-6)
    np.testing.assert_array_equal(g["phi"], sim.fields(("phi",))["phi"])
    fg, fo = sim.force(40.0, 40.0), o.force(40.0, 40.0)
    assert abs(fg[0] - fo[0]) <= 1e-4 * abs(fo[0])
    assert abs(fg[1] - fo[1]) <= 1e-4 * abs(fo[0])
    assert abs(fg[2] - fo[2]) <= 1e-4 * abs(fo[0]) * 8.0
    assert sim.steps == 0


def recirculation_length(ux_row, x_rear):
    """Distance from the cylinder's rear to the first sign change of u_x
    (negative to positive) on the wake centre line, linearly interpolated."""
    x0 = int(np.ceil(x_rear))
    for x in range(x0, len(ux_row) - 1):
        if ux_row[x] < 0.0 <= ux_row[x + 1]:
            return x + ux_row[x] / (ux_row[x] - ux_row[x + 1]) - x_rear
    return float("nan")


def run_cylinder(lbm, Re, max_steps=200_000, chunk=10_000):
    c = W.cylinder_flow(Re=Re)
    cx, cy, R = (float(v) for v in c.seeds[0, :3])
    sim = lbm.Simulation(c.params)
    sim.init_seeds(c.seeds, c.U0, c.theta0)
    u0 = 0.1
    cds, done = [], 0
    while done < max_steps:
        sim.step_flow(chunk)
        done += chunk
        fx = sim.force(cx, cy)[0]
        cds.append(fx / (R * u0 * u0))
        if len(cds) > 3 and abs(cds[-1] - cds[-2]) <= 1e-4 * abs(cds[-1]):
            break
    ux = sim.fields(("ux",))["ux"]
    lw = recirculation_length(ux[int(round(cy))], cx + R) / R
    return cds[-1], lw, done, cds


# Table 1 of the paper ("present" row).  The published values for the same
# flows spread by 1 % (Re 20) to 7 % (Re 40) in C_d and 3 % in L_W; the bounds
# allow 5 % on C_d and 10 % on L_W, whose end point on a diffuse surface is
# only defined to about one interface width (0.05 R here).
@pytest.mark.parametrize("Re,cd_paper,lw_paper", [(20.0, 2.153, 1.853), (40.0, 1.598, 4.491)])
def test_cylinder_drag_and_wake_against_table1(lbm, Re, cd_paper, lw_paper):
    cd, lw, steps, hist = run_cylinder(lbm, Re)
    print(f"Re {Re}: C_d {cd:.4f} (paper {cd_paper}), L_W {lw:.3f} (paper {lw_paper}) after {steps} flow steps; "
          f"C_d history {[round(v, 4) for v in hist]}")
    assert abs(cd - cd_paper) <= 0.05 * cd_paper
    assert abs(lw - lw_paper) <= 0.10 * lw_paper
