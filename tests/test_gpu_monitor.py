"""Periodic reductions inside lbm_step (the device metrics ring) against
metrics taken by hand at the same steps, and the tip velocities against
finite differences of the recorded tips."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2209_01444_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_2209_01444_gb300 import build_ext, lbm as L

    build_ext.build()
    L.load()
    return L


def _sim(L):
    c = workloads.single_seed_periodic(96)
    s = L.Simulation(c.params)
    s.init_seeds(c.seeds, c.U0, c.theta0)
    return s, c


@pytest.mark.parametrize("every", [50, 37])
def test_monitor_records_match_metrics(lbm, every):
    a, c = _sim(lbm)
    cx, cy = float(c.seeds[0, 0]), float(c.seeds[0, 1])
    a.set_monitor(every, 8, cx, cy)
    a.step(400)
    recs = a.monitor()
    n_total = 400 // every + 1
    assert len(recs) == min(8, n_total)
    steps = [r["step"] for r in recs]
    assert steps == [every * k for k in range(n_total - len(recs), n_total)]
    b, _ = _sim(lbm)
    done = 0
    for r in recs:
        b.step(r["step"] - done)
        done = r["step"]
        m = b.metrics(cx, cy)
        for k in ("tip_px", "tip_mx", "tip_py", "solid_fraction", "sum_C", "sum_H", "sum_h", "sum_phi"):
            assert m[k] == r[k], (k, m[k], r[k])
    # tip velocities: finite differences of consecutive records in W0 / tau0
    dt = c.params["dt"]
    assert math.isnan(recs[0]["v_px"]) == (n_total > 8)
    for p, q in zip(recs, recs[1:]):
        v = (q["tip_px"] - p["tip_px"]) * c.params["dx"] / ((q["step"] - p["step"]) * dt)
        assert abs(q["v_px"] - v) <= 1e-12 * max(1.0, abs(v))
    assert recs[-1]["v_px"] > 0  # the seed grows


def test_monitor_off_and_bad_arguments(lbm):
    a, c = _sim(lbm)
    with pytest.raises(lbm.LBMError):
        a.set_monitor(10, 1, 0.0, 0.0)
    a.set_monitor(0, 0, 0.0, 0.0)
    a.step(20)
    assert a.monitor() == []
