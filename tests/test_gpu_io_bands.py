"""Whole-grid transfers through the bounded band buffer: any band size gives
the same result bit for bit, and a handle holds only its state, so the
largest grids the device can hold run."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2209_01444_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    from paper_2209_01444_gb300 import build_ext, lbm as L

    build_ext.build()
    L.load()
    return L


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_one_row_bands_equal_the_default(lbm, storage):
    """45 x 37 random fields (init_fields), 37 x 29 seeds (init_seeds): with a
    1-byte limit every transfer goes one row at a time."""
    nx, ny = 45, 37
    p = W.thermosolutal_params(nx, ny, bc=("inflow", "outflow", "noslip", "symmetry"), u_in=(0.15, 0.02),
                               gbetaT=W.GBETA_T * 5, theta_ref=-0.5, dir_theta=-0.4)
    f, orient = W.random_fields(nx, ny, rng_seed=77)
    sims = []
    for chunk in (None, 1):
        s = lbm.Simulation(p, storage)
        if chunk:
            s.set_io_chunk(chunk)
        s.init_fields(f, orient)
        s.step(11)
        sims.append(s)
    a, b = sims
    np.testing.assert_array_equal(a.state(), b.state())
    fa, fb = a.fields(), b.fields()
    for k in fa:
        np.testing.assert_array_equal(fa[k], fb[k])
    np.testing.assert_array_equal(a.state_region(3, 5, 20, 17), b.state_region(3, 5, 20, 17))
    st = a.state()
    st[:, 4, 7] *= 1.0001
    b.set_state(st)
    a.set_state(st)
    np.testing.assert_array_equal(a.state(), b.state())
    q = W.thermosolutal_params(37, 29)
    seeded = []
    for chunk in (None, 1):
        s = lbm.Simulation(q, storage)
        if chunk:
            s.set_io_chunk(chunk)
        s.init_seeds(np.array([[18.0, 14.0, 6.0, 0.3], [5.0, 5.0, 3.0, 0.1]]), -0.2, -0.5)
        seeded.append(s.state())
    np.testing.assert_array_equal(*seeded)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_fp32_fields_are_the_fp64_fields_rounded(lbm, storage):
    """lbm_get_fields_f32 on a 45 x 37 grid (row pitch 64): phi, C, U and theta
    (offsets of -1, +1, 0 and theta_ref added to FP32 deviations) are the FP64
    fields rounded to FP32 exactly; u_x, u_y and p carry one more rounding (of
    their FP32 scale factor), within 2 units in the last place.  One-row bands,
    page-locked output and a subset of the fields give the same values."""
    import torch

    nx, ny = 45, 37
    p = W.thermosolutal_params(nx, ny, bc=("inflow", "outflow", "noslip", "symmetry"), u_in=(0.15, 0.02),
                               gbetaT=W.GBETA_T * 5, theta_ref=-0.5, dir_theta=-0.4)
    f, orient = W.random_fields(nx, ny, rng_seed=78)
    s = lbm.Simulation(p, storage)
    s.init_fields(f, orient)
    s.step(11)
    want = s.fields()
    got = s.fields_f32()  # pageable output, default bands
    for k in ("phi", "C", "U", "theta"):
        np.testing.assert_array_equal(got[k], want[k].astype(np.float32), err_msg=k)
    for k in ("ux", "uy", "p"):
        np.testing.assert_array_max_ulp(got[k], want[k].astype(np.float32), maxulp=2)
    pinned = torch.empty((2, ny, nx), dtype=torch.float32, pin_memory=True).numpy()
    s.set_io_chunk(1)
    for out in (pinned, None):  # page-locked: direct copies; pageable: staged, one row per band
        sub = s.fields_f32(("uy", "theta"), out=out)
        assert list(sub) == ["theta", "uy"]
        np.testing.assert_array_equal(sub["theta"], got["theta"])
        np.testing.assert_array_equal(sub["uy"], got["uy"])
    np.testing.assert_array_equal(pinned[1], got["uy"])


def test_largest_grid_that_fits(lbm):
    """FP16 storage on the largest square grid within 75 % of the free device
    memory (below 2^31 nodes): seeds, 4 steps and the metrics, all on the
    device; every node stays finite and the solute sum holds to 1e-4.  (FP16
    keeps 11 bits of each moving population deviation; in a uniform melt at
    U0 = -0.55 every node rounds alike, so the sum moves coherently, by a
    fraction of 2^-11 of the deviation mass, not as a random walk.)"""
    import torch

    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    per_node = 2 * (12 * 2 + 3 * 4 + 9 * 2) + 6 * 4 + 1  # state bytes per node, FP16 storage
    nodes = min(0.75 * free / per_node, 2.0**31 - 2.0**27)
    n = int(math.sqrt(nodes)) // 32 * 32
    assert n >= 4096
    p = W.thermosolutal_params(n, n, eps_s=0.05)
    s = lbm.Simulation(p, "fp16")
    c = n / 2
    s.init_seeds(np.array([[c, c, 12.0, 0.0]]), -0.55, -0.55)
    m0 = s.metrics(c, c)
    s.step(4)
    m1 = s.metrics(c, c)
    print(f"{n} x {n} = {n * n / 1e9:.2f} G nodes, FP16; tip {m0['tip_px']:.2f} -> {m1['tip_px']:.2f}; "
          f"sum C drift {(m1['sum_C'] - m0['sum_C']) / m0['sum_C']:.2e}")
    assert m1["nonfinite"] == 0
    assert abs(m1["sum_C"] - m0["sum_C"]) <= 1e-4 * abs(m0["sum_C"])
    assert abs(m0["tip_px"] - 12.0) < 0.5 and m1["tip_px"] > 0
