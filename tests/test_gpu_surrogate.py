"""The surrogate coupled to the LB solver on the GPU: device-side field
exchange, snapshots, one surrogate window with and without the LB audit, and
training on trajectories the LB itself generates."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import unet_oracle as U
from paper_2209_01444_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2209_01444_gb300 import build_ext, lbm, surrogate

    build_ext.build()
    lbm.load()
    torch.cuda.init()
    return torch, lbm, surrogate


def _sim(lbm, n=64, steps=200):
    c = workloads.forced_flow(n, u_lattice=0.01)
    c.seeds[:, 2] = 6.0
    sim = lbm.Simulation(c.params)
    sim.init_seeds(c.seeds, c.U0, c.theta0)
    sim.step(steps)
    return sim, c


def test_fields_nhwc_match_get_fields(env):
    torch, lbm, S = env
    sim, _ = _sim(lbm)
    got = sim.fields_nhwc().cpu().numpy().astype(np.float64)
    ref = sim.fields(("phi", "C", "theta", "ux", "uy"))
    for k, name in enumerate(("phi", "C", "theta", "ux", "uy")):
        r = ref[name]
        assert np.abs(got[..., k] - r).max() <= 1e-6 * max(np.abs(r).max(), 1e-3), name


def test_set_fields_round_trip_and_snapshots(env):
    torch, lbm, S = env
    sim, _ = _sim(lbm)
    state0 = sim.state()
    f0 = sim.fields_nhwc().clone()
    sim.snapshot_save(0)
    p0 = sim.fields(("p",))["p"]
    sim.set_fields_nhwc(f0)
    f1 = sim.fields_nhwc()
    d = (f1 - f0).abs().amax(dim=(0, 1)).cpu().numpy()
    scale = f0.abs().amax(dim=(0, 1)).cpu().numpy()
    assert np.all(d <= 1e-5 * np.maximum(scale, 1e-3)), (d, scale)  # velocity included
    p1 = sim.fields(("p",))["p"]
    assert np.abs(p1 - p0).max() <= 1e-4 * max(np.abs(p0).max(), 1e-6)
    n0 = sim.steps
    sim.step(20)
    assert np.isfinite(sim.fields_nhwc().cpu().numpy()).all()
    sim.snapshot_restore(0)
    assert sim.steps == n0
    np.testing.assert_array_equal(sim.state(), state0)


def _identity_net(S, torch, n):
    net = S.UNet(1, n, n)
    p = workloads.unet_params(S.param_shapes(), 7)
    p["out.W"][:] = 0.0
    p["out.b"][:] = 0.0
    net.set_params(p)
    return net


def test_surrogate_window_and_audit(env):
    """With a zero output projection the network predicts no change; an
    unaudited window then leaves the equilibrium of the old fields, an audited
    one keeps exactly the plain LB result and reports the tip movement."""
    torch, lbm, S = env
    sim, c = _sim(lbm)
    net = _identity_net(S, torch, 64)
    cx, cy = float(c.seeds[0, 0]), float(c.seeds[0, 1])
    ref, _ = _sim(lbm)
    ref.step(50)
    tips_lb = ref.metrics(cx, cy)
    f0 = sim.fields_nhwc().clone()
    tips0 = sim.metrics(cx, cy)
    sim.snapshot_save(0)
    rep = sim.surrogate_advance(net, 50, 1.0, True, cx, cy)
    assert rep["audited"]
    np.testing.assert_array_equal(sim.state(), ref.state())
    assert sim.steps == ref.steps
    moved = max(abs(tips_lb[k] - tips0[k]) for k in ("tip_px", "tip_mx", "tip_py"))
    assert abs(rep["tip_err"] - moved) <= 0.05 + 0.05 * moved, (rep, moved)
    assert rep["accepted"] == (rep["tip_err"] <= 1.0)
    assert rep["mismatch"] >= 0 and rep["max_dphi"] >= 0.0
    sim.snapshot_restore(0)
    n0 = sim.steps
    rep = sim.surrogate_advance(net, 50, 1.0, False, cx, cy)
    assert not rep["audited"] and sim.steps == n0 + 50
    f1 = sim.fields_nhwc()
    assert float((f1 - f0).abs().max()) <= 1e-4


def test_prediction_that_is_not_finite_is_never_applied(env):
    """A network whose output is not finite (here a NaN output bias): an
    unaudited window leaves the state and the step count as they were and
    reports the window as not accepted; an audited one keeps the plain LB
    result and rejects the prediction."""
    torch, lbm, S = env
    sim, c = _sim(lbm)
    net = S.UNet(1, 64, 64)
    p = workloads.unet_params(S.param_shapes(), 7)
    p["out.b"][:] = np.nan
    net.set_params(p)
    cx, cy = float(c.seeds[0, 0]), float(c.seeds[0, 1])
    state0, n0 = sim.state(), sim.steps
    rep = sim.surrogate_advance(net, 50, 1.0, False, cx, cy)
    assert not rep["audited"] and not rep["accepted"] and rep["tip_err"] == float("inf")
    assert sim.steps == n0
    np.testing.assert_array_equal(sim.state(), state0)
    ref, _ = _sim(lbm)
    ref.step(50)
    rep = sim.surrogate_advance(net, 50, 1.0, True, cx, cy)
    assert rep["audited"] and not rep["accepted"]
    np.testing.assert_array_equal(sim.state(), ref.state())


def test_training_on_lb_trajectories_beats_persistence(env):
    """A network trained for 500 steps on (t, t + 50) pairs of LB runs
    predicts the pairs of a held-out domain better than 'no change'."""
    torch, lbm, S = env
    cases = workloads.surrogate_domains(count=6, n=64, rng_seed=9)
    x, t = S.make_dataset(cases, K=50, windows=10, warm=100)
    n = x.shape[0]
    hold = np.arange(n) % 6 == 5  # the last domain is held out
    xs, ts = x[torch.from_numpy(~hold).cuda()], t[torch.from_numpy(~hold).cuda()]
    xh, th = x[torch.from_numpy(hold).cuda()], t[torch.from_numpy(hold).cuda()]
    mean, std_in, std_out = S.normalisation(xs, ts)
    net = S.UNet(4, 64, 64)
    net.set_params(workloads.unet_params(S.param_shapes(), 3))
    net.set_norm(mean, std_in, std_out)
    S.train(net, xs, ts, steps=500, lr=1e-3, seed=1)
    ev = S.UNet(xh.shape[0], 64, 64)
    ev.set_params(net.params())
    ev.set_norm(mean, std_in, std_out)
    pred = ev.forward(xh.contiguous())
    sd = torch.from_numpy(std_out).cuda()
    err_net = float((((pred - th) / sd) ** 2).mean())
    err_persist = float((((xh - th) / sd) ** 2).mean())
    print(f"held-out normalised MSE: network {err_net:.4e}, persistence {err_persist:.4e}")
    assert np.isfinite(err_net) and err_net < 0.8 * err_persist
