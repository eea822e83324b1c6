"""The batched persistent launch against single-domain handles and the oracle.

Domains of uneven sizes (ragged tiles), wall types and parameters advance
together; each must evolve exactly as it does alone."""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import oracle as O
import storage_emulation as SE
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
    """Each domain of the batched launch evolves as it does alone in the
    single-domain kernel.  Both run the same per-node code, inlined into
    kernels with different tile heights, where the compiler may fuse a
    product into a multiply-add differently: the fields agree to FP32
    rounding grown over 37 steps (1e-5 of each field's scale; U, which
    multiplies solute differences by up to 16 in the solid, shows the
    largest, about 2e-6).  A misplaced load or store moves a field by O(0.1)."""
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
            assert np.abs(got[k] - want[k]).max() <= 1e-5 * scale, (j, k)


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


# ------------------------------------------------------------ FP16 storage
def errors(got, want, theta0):
    """The parity metric: max|X - X_ref| / max(max|X_ref|, floor), floors phi,
    C: 1, theta: |theta0|.  The velocity components share one scale, the
    largest speed |u| of the reference (floor 1e-6): the tolerance reading's u
    floor is that of the velocity, so a cross-stream component that is still
    small next to the stream is not measured against its own tiny maximum."""
    out = {}
    for k, fl in (("phi", 1.0), ("C", 1.0), ("theta", abs(theta0))):
        out[k] = float(np.abs(got[k] - want[k]).max() / max(np.abs(want[k]).max(), fl))
    speed = max(float(np.hypot(want["ux"], want["uy"]).max()), 1e-6)
    for k in ("ux", "uy"):
        out[k] = float(np.abs(got[k] - want[k]).max() / speed)
    return out


ACC = ("phi", "C", "theta", "ux", "uy")


@pytest.mark.parametrize("ty,run", [(4, 1), (8, 1), (16, 0)])
def test_fp16_batch_matches_fp16_single_domain_runs(lbm, ty, run):
    """The batched kernel with FP16 storage against each domain stepped alone
    by the single-domain FP16 kernel: the same per-node arithmetic and the
    same rounding of every stored population, so the two agree to a few
    units of the 16-bit rounding (a product fused into a multiply-add
    differently by the compiler can move a value across a rounding boundary)."""
    cases = small_cases()
    b = lbm.Batch([c.params for c in cases], "fp16")
    b.set_tiling(ty, run)
    singles = []
    for j, c in enumerate(cases):
        b.init_seeds(j, c.seeds, c.U0, c.theta0)
        s = lbm.Simulation(c.params, "fp16")
        s.init_seeds(c.seeds, c.U0, c.theta0)
        singles.append(s)
    b.step(37)           # two 16-step graphs + 5 direct steps
    worst = {}
    for j, (c, s) in enumerate(zip(cases, singles)):
        s.step(37)
        e = errors(b.fields(j, ACC), s.fields(ACC), c.theta0)
        print(j, {k: f"{v:.1e}" for k, v in e.items()})
        for k, v in e.items():
            worst[k] = max(worst.get(k, 0.0), v)
    assert max(worst.values()) <= 1e-3, worst


def test_fp16_batch_matches_the_oracle_with_fp16_storage(lbm):
    """The FP16 batched launch against the FP64 oracle whose state is rounded
    after every step as FP16 storage rounds it (within 2e-3: the kernels'
    FP32 arithmetic against FP64, amplified by nothing), and against the plain
    oracle within the 16-bit bound of 1e-2."""
    cases = small_cases()[:4]
    b = lbm.Batch([c.params for c in cases], "fp16")
    for j, c in enumerate(cases):
        b.init_seeds(j, c.seeds, c.U0, c.theta0)
    steps = 60
    b.step(steps)
    for j, c in enumerate(cases):
        o, r = O.Oracle(c.params), O.Oracle(c.params)
        o.init_seeds(c.seeds, c.U0, c.theta0)
        r.init_seeds(c.seeds, c.U0, c.theta0)
        SE.round_state(r, c.params, "fp16")
        o.step(steps)
        for _ in range(steps):
            r.step(1)
            SE.round_state(r, c.params, "fp16")
        got = b.fields(j, ACC)
        vs_rounded, vs_plain = errors(got, r.fields(), c.theta0), errors(got, o.fields(), c.theta0)
        print(j, {k: f"{vs_rounded[k]:.1e} / {vs_plain[k]:.1e}" for k in ACC})
        assert max(vs_rounded.values()) <= 2e-3, (j, vs_rounded, vs_plain)
        assert max(vs_plain.values()) <= 1e-2, (j, vs_rounded, vs_plain)


def test_fp16_batch_of_the_sweep_matches_the_oracle(lbm):
    """The 256-domain parameter sweep (sides log-uniform in 128..1024, the
    benchmarked batched FP16 launch with its 16-step graphs) on its smallest
    domain (130 x 130, inflow u_x = 0.27 W0/tau0) against the FP64 oracle,
    after 32 steps (the flow still starting impulsively, its cross-stream
    component small) and 516 steps: within 2e-3 of the oracle rounded as
    FP16 storage rounds it, and within 1e-2 of the plain oracle.  The
    cross-stream velocity measured against its own maximum is reported too:
    that is where the FP16 format itself departs most from FP64."""
    cases = W.batch_domains()
    j = min(range(len(cases)), key=lambda i: cases[i].nodes)
    c = cases[j]
    b = lbm.Batch([q.params for q in cases], "fp16")
    for i, q in enumerate(cases):
        b.init_seeds(i, q.seeds, q.U0, q.theta0)
    o, r = O.Oracle(c.params), O.Oracle(c.params)
    o.init_seeds(c.seeds, c.U0, c.theta0)
    r.init_seeds(c.seeds, c.U0, c.theta0)
    SE.round_state(r, c.params, "fp16")
    for T in (32, 516):
        b.step(T - o.steps)
        for _ in range(T - o.steps):
            o.step(1)
            r.step(1)
            SE.round_state(r, c.params, "fp16")
        got, want, rw = b.fields(j, ACC), o.fields(), r.fields()
        vs_rounded, vs_plain = errors(got, rw, c.theta0), errors(got, want, c.theta0)
        own = float(np.abs(got["uy"] - want["uy"]).max() / np.abs(want["uy"]).max())
        fmt = float(np.abs(rw["uy"] - want["uy"]).max() / np.abs(want["uy"]).max())
        print(T, {k: f"{vs_rounded[k]:.1e} / {vs_plain[k]:.1e}" for k in ACC},
              f"uy of its own max: gpu {own:.2e}, rounded oracle {fmt:.2e}")
        assert max(vs_rounded.values()) <= 2e-3, (T, vs_rounded, vs_plain)
        assert max(vs_plain.values()) <= 1e-2, (T, vs_rounded, vs_plain)
        assert b.metrics(j, *c.seeds[0][:2], c.seeds[0][3])["tip_px"] == pytest.approx(
            o.metrics(*c.seeds[0][:2], c.seeds[0][3])["tip_px"], abs=1.0)


def test_batch_kernel_timing_runs_direct_steps_and_keeps_the_state(lbm):
    """lbm_batch_set_profiling: timed steps launch the batched kernel directly
    (one timed launch per step) and give the state graph replay gives, to
    16-bit rounding (inside the step graphs the left/right walls are updated
    as the next step loads them, in direct launches by the column pass: the
    same arithmetic in another kernel, rounded once more or once less)."""
    cases = small_cases()[:3]
    out = []
    for prof in (False, True):
        b = lbm.Batch([c.params for c in cases], "fp16")
        for j, c in enumerate(cases):
            b.init_seeds(j, c.seeds, c.U0, c.theta0)
        b.set_profiling(prof)
        b.step(20)
        if prof:
            ms, n = b.kernel_time()
            assert n == 20 and ms > 0
            b.set_profiling(False)
            assert b.kernel_time() == (0.0, 0)
        out.append([b.fields(j, ACC) for j in range(len(cases))])
    for a, c, case in zip(*out, cases):
        e = errors(a, c, case.theta0)
        assert max(e.values()) <= 4e-3, e
