"""The batched persistent launch against single-domain handles and the oracle.

Domains of uneven sizes (ragged tiles), wall types and parameters advance
together; each must evolve exactly as it does alone."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2209_01444_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch

    from paper_2209_01444_gb300 import build_ext, lbm as L

    build_ext.build()
    L.load()
    torch.cuda.init()
    return L


def small_cases():
    """Five small domains covering ragged sizes, every wall family, grain
    rotation and inflow speeds, in the parameter ranges of the batch sweep."""
    cases = []
    shapes = [(40, 33), (64, 64), (100, 47), (37, 90), (72, 72)]
    bcs = [("periodic",) * 4, ("inflow", "outflow", "symmetry", "symmetry"), ("periodic", "periodic", "noslip", "noslip"),
           ("inflow", "outflow", "symmetry", "symmetry"), ("dirichlet",) * 4]
    for j, ((nx, ny), bc) in enumerate(zip(shapes, bcs)):
        delta = 0.3 + 0.1 * j
        p = W.thermosolutal_params(nx, ny, eps_s=0.02 + 0.01 * j, theta_ref=-delta, bc=bc,
                                   u_in=(0.1 * j, 0.0), dir_theta=-delta)
        seeds = np.array([[0.375 * nx, 0.5 * ny, 6.0, math.pi / 4 * j / 5]])
        cases.append(W.Case(f"d{j}", p, seeds, 0.0, -delta, 40))
    return cases


@pytest.mark.parametrize("ty,run", [(4, 1), (8, 1), (16, 1), (8, 4), (4, 0), (16, 0)])
def test_batch_matches_single_domain_runs(lbm, ty, run):
    cases = small_cases()
    b = lbm.Batch([c.params for c in cases])
    b.set_tiling(ty, run)
    singles = []
    for j, c in enumerate(cases):
        b.init_seeds(j, c.seeds, c.U0, c.theta0)
        s = lbm.Simulation(c.params)
        s.init_seeds(c.seeds, c.U0, c.theta0)
        singles.append(s)
    b.step(37)           # two 16-step graphs + 5 direct steps
    for j, (c, s) in enumerate(zip(cases, singles)):
        s.step(37)
        got, want = b.fields(j), s.fields()
        for k in want:
            scale = max(np.abs(want[k]).max(), 1e-6)
            assert np.abs(got[k] - want[k]).max() <= 1e-6 * scale, (j, k)


def test_batch_matches_the_oracle(lbm):
    cases = small_cases()[:2]
    b = lbm.Batch([c.params for c in cases])
    for j, c in enumerate(cases):
        b.init_seeds(j, c.seeds, c.U0, c.theta0)
    b.step(60)
    for j, c in enumerate(cases):
        o = O.Oracle(c.params)
        o.init_seeds(c.seeds, c.U0, c.theta0)
        o.step(60)
        want, got = o.fields(), b.fields(j)
        for k, fl in (("phi", 1.0), ("C", 1.0), ("theta", abs(c.theta0)), ("ux", 1e-6), ("uy", 1e-6)):
            err = np.abs(got[k] - want[k]).max() / max(np.abs(want[k]).max(), fl)
            assert err <= 1e-4, (j, k, err)
        mg, mo = b.metrics(j, *c.seeds[0][:2], c.seeds[0][3]), o.metrics(*c.seeds[0][:2], c.seeds[0][3])
        assert mg["tip_px"] == pytest.approx(mo["tip_px"], abs=2e-3)


def test_tuning_picks_a_height_and_leaves_the_state(lbm, tmp_path):
    cases = small_cases()
    b = lbm.Batch([c.params for c in cases])
    for j, c in enumerate(cases):
        b.init_seeds(j, c.seeds, c.U0, c.theta0)
    b.step(5)
    before = [b.fields(j) for j in range(len(cases))]
    cache = str(tmp_path / "tiles.txt")
    ty = b.tune(cache)
    assert ty in (4, 8, 16) and b.tile_height == ty
    after = [b.fields(j) for j in range(len(cases))]
    for x, y in zip(before, after):
        for k in x:
            np.testing.assert_array_equal(x[k], y[k])
    assert open(cache).read().split()[-2:] == [str(ty), str(b.tiles_per_cta)]
    b2 = lbm.Batch([c.params for c in cases])
    for j, c in enumerate(cases):
        b2.init_seeds(j, c.seeds, c.U0, c.theta0)
    assert b2.tune(cache) == ty          # served from the cache
    assert len(open(cache).read().splitlines()) == 1


def test_batch_rejects_mixed_storage(lbm):
    cases = small_cases()[:2]
    lib = lbm.load()
    arr = (lbm.lbm_params * 2)(lbm.make_params(cases[0].params, "fp32"), lbm.make_params(cases[1].params, "fp16"))
    import ctypes as ct
    h = ct.c_void_p()
    assert lib.lbm_batch_create(arr, 2, ct.byref(h)) == lbm.LBM_EINVAL
    assert b"storage" in lib.lbm_batch_last_error(None)
