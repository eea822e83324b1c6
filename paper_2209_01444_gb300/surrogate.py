"""Binding of the surrogate network (``lbm_unet_*`` in ``include/lbm.h``).

Argument marshalling only: the forward pass, the loss, the backward pass and
the Adam update all run in the library's CUDA kernels.  Tensors passed in are
CUDA ``torch.float32`` arrays of shape [batch, height, width, fields]; torch is
used for device memory and streams only.
"""
from __future__ import annotations

import ctypes as ct
import os
import math

import numpy as np

from . import lbm as L

# The network the surrogate runs: five levels of widths 32 .. 512 and five
# fields (phi, C, theta, u_x, u_y) in and out.
LEVELS = 5
BASE = 32
FIELDS = ("phi", "C", "theta", "ux", "uy")
IN_PITCH = 8  # input channels as the first convolution sees them (fields, zero padded)


def param_shapes(levels: int = LEVELS, base: int = BASE, fields: int = len(FIELDS)):
    """(name, shape) of every parameter tensor, in the library's order."""
    shapes = []
    c_prev = IN_PITCH
    for l in range(levels):
        c = base << l
        shapes += [(f"enc{l}a.W", (c, 9 * c_prev)), (f"enc{l}a.b", (c,)),
                   (f"enc{l}b.W", (c, 9 * c)), (f"enc{l}b.b", (c,))]
        c_prev = c
    for l in range(levels - 2, -1, -1):
        c = base << l
        shapes += [(f"up{l}.W", (4 * c, 2 * c)), (f"up{l}.b", (4 * c,)),
                   (f"dec{l}a.W", (c, 18 * c)), (f"dec{l}a.b", (c,)),
                   (f"dec{l}b.W", (c, 9 * c)), (f"dec{l}b.b", (c,))]
    shapes += [("out.W", (fields, base)), ("out.b", (fields,))]
    return shapes


def flatten(params: dict, shapes) -> np.ndarray:
    return np.concatenate([np.asarray(params[n], np.float32).reshape(-1) for n, _ in shapes])


def unflatten(vec: np.ndarray, shapes) -> dict:
    out, o = {}, 0
    for n, shp in shapes:
        k = int(np.prod(shp))
        out[n] = vec[o:o + k].reshape(shp)
        o += k
    return out


class UNet:
    """The network sized for `batch` images of height x width pixels."""

    def __init__(self, batch: int, height: int, width: int, levels: int = LEVELS, base: int = BASE,
                 fields: int = len(FIELDS), stream=None):
        self.lib = L.load()
        h = ct.c_void_p()
        rc = self.lib.lbm_unet_create(levels, base, fields, batch, height, width, ct.byref(h))
        if rc != L.LBM_OK:
            raise L.LBMError(rc, f"lbm_unet_create({levels}, {base}, {fields}, {batch}, {height}, {width})")
        self.h = h
        self.levels, self.base, self.fields = levels, base, fields
        self.shape = (batch, height, width, fields)
        self.shapes = param_shapes(levels, base, fields)
        if stream is not None:
            self.set_stream(stream)

    def __del__(self):
        h, self.h = getattr(self, "h", None), None
        if h:
            self.lib.lbm_unet_destroy(h)

    def _check(self, rc: int) -> None:
        if rc != L.LBM_OK:
            raise L.LBMError(rc, (self.lib.lbm_unet_last_error(self.h) or b"").decode())

    def _t(self, t):
        import torch

        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous(), "CUDA float32 contiguous expected"
        assert tuple(t.shape) == self.shape, (tuple(t.shape), self.shape)
        return ct.c_void_p(t.data_ptr())

    def set_stream(self, stream) -> None:
        raw = getattr(stream, "cuda_stream", stream)
        self._check(self.lib.lbm_unet_set_stream(self.h, ct.c_void_p(raw or 0)))

    @property
    def param_count(self) -> int:
        return int(self.lib.lbm_unet_param_count(self.h))

    @property
    def device_bytes(self) -> int:
        return int(self.lib.lbm_unet_device_bytes(self.h))

    def set_params(self, params) -> None:
        vec = flatten(params, self.shapes) if isinstance(params, dict) else np.asarray(params, np.float32)
        vec = np.ascontiguousarray(vec, np.float32)
        assert vec.size == self.param_count
        self._check(self.lib.lbm_unet_set_params(self.h, vec.ctypes.data_as(ct.c_void_p)))

    def _get(self, fn) -> dict:
        vec = np.empty(self.param_count, np.float32)
        self._check(fn(self.h, vec.ctypes.data_as(ct.c_void_p)))
        return unflatten(vec, self.shapes)

    def params(self) -> dict:
        return self._get(self.lib.lbm_unet_get_params)

    def grads(self) -> dict:
        return self._get(self.lib.lbm_unet_get_grads)

    def set_norm(self, mean, std_in, std_out=None) -> None:
        """Inputs read as (x - mean) / std_in; the output is the increment in
        units of std_out (default std_in)."""
        m = np.ascontiguousarray(mean, np.float32)
        si = np.ascontiguousarray(std_in, np.float32)
        so = si if std_out is None else np.ascontiguousarray(std_out, np.float32)
        assert m.size == self.fields and si.size == self.fields and so.size == self.fields
        self._check(self.lib.lbm_unet_set_norm(self.h, m.ctypes.data_as(ct.c_void_p), si.ctypes.data_as(ct.c_void_p),
                                               so.ctypes.data_as(ct.c_void_p)))
        self.norm = (m, si, so)

    def set_loss_weight(self, alpha: float) -> None:
        """Interface weight of the loss: squared errors at each pixel weighted
        by 1 + alpha max(0, 1 - phi^2), phi the input's phase field."""
        self._check(self.lib.lbm_unet_set_loss_weight(self.h, float(alpha)))
        self.loss_weight = float(alpha)

    def save(self, path: str) -> None:
        """Parameters and normalisation to a weight file (lbm_unet_save)."""
        self._check(self.lib.lbm_unet_save(self.h, os.fsencode(path)))

    def load(self, path: str) -> None:
        """Parameters and normalisation from a weight file of a network of the
        same levels, base and fields (lbm_unet_load)."""
        self._check(self.lib.lbm_unet_load(self.h, os.fsencode(path)))

    def forward(self, x, y=None):
        """Prediction in physical units (into `y` when given)."""
        import torch

        if y is None:
            y = torch.empty_like(x)
        self._check(self.lib.lbm_unet_forward(self.h, self._t(x), self._t(y)))
        return y

    def output_normalised(self):
        """The last network output, the increment in units of std_out (a new
        CUDA tensor)."""
        import torch

        out = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        self._check(self.lib.lbm_unet_output(self.h, self._t(out)))
        return out

    def backward(self, x, target) -> None:
        self._check(self.lib.lbm_unet_backward(self.h, self._t(x), self._t(target)))

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8) -> None:
        self._check(self.lib.lbm_unet_adam(self.h, lr, beta1, beta2, eps))

    def train_step(self, x, target, lr: float) -> None:
        self._check(self.lib.lbm_unet_train_step(self.h, self._t(x), self._t(target), lr))

    def loss(self) -> float:
        out = ct.c_double()
        self._check(self.lib.lbm_unet_loss(self.h, ct.byref(out)))
        return out.value


# ---------------------------------------------------------------- training
def make_snapshots(cases, K: int, windows: int, warm: int = 0, storage: str = "fp32"):
    """Runs the cases (equal grid sizes) as one batched LB launch and records
    the fields every K steps after `warm` steps: a device tensor
    [windows + 1, len(cases), ny, nx, 5]."""
    import torch

    ny, nx = int(cases[0].params["ny"]), int(cases[0].params["nx"])
    assert all(int(c.params["ny"]) == ny and int(c.params["nx"]) == nx for c in cases)
    b = L.Batch([c.params for c in cases], storage=storage)
    for d, c in enumerate(cases):
        b.init_seeds(d, c.seeds, c.U0, c.theta0)
    if warm:
        b.step(warm)
    D = len(cases)
    snaps = torch.empty(windows + 1, D, ny, nx, 5, dtype=torch.float32, device="cuda")
    for w in range(windows + 1):
        for d in range(D):
            b.fields_nhwc(d, snaps[w, d])
        if w < windows:
            b.step(K)
    b.synchronize()
    return snaps


def make_dataset(cases, K: int, windows: int, warm: int = 0, storage: str = "fp32"):
    """Runs the cases (equal grid sizes) as one batched LB launch and records
    the fields every K steps after `warm` steps.  Returns device tensors x, t
    [windows * len(cases), ny, nx, 5] of consecutive snapshots (t is x advanced
    by K steps)."""
    import torch

    ny, nx = int(cases[0].params["ny"]), int(cases[0].params["nx"])
    assert all(int(c.params["ny"]) == ny and int(c.params["nx"]) == nx for c in cases)
    b = L.Batch([c.params for c in cases], storage=storage)
    for d, c in enumerate(cases):
        b.init_seeds(d, c.seeds, c.U0, c.theta0)
    if warm:
        b.step(warm)
    D = len(cases)
    snaps = torch.empty(windows + 1, D, ny, nx, 5, dtype=torch.float32, device="cuda")
    for w in range(windows + 1):
        for d in range(D):
            b.fields_nhwc(d, snaps[w, d])
        if w < windows:
            b.step(K)
    b.synchronize()
    x = snaps[:-1].reshape(windows * D, ny, nx, 5)
    t = snaps[1:].reshape(windows * D, ny, nx, 5)
    return x, t


def normalisation(x, t, floor: float = 1e-6):
    """Per-field mean and standard deviation of the inputs, and the standard
    deviation of the K-step increments (so that every field's increment
    weighs alike in the loss)."""
    step = max(1, x.shape[0] // 64)
    xs = x[::step].cpu().numpy().astype(np.float64).reshape(-1, 5)
    ds = t[::step].cpu().numpy().astype(np.float64).reshape(-1, 5) - xs
    mean = xs.mean(axis=0)
    std_in = np.maximum(xs.std(axis=0), floor)
    std_out = np.maximum(ds.std(axis=0), floor)
    return mean.astype(np.float32), std_in.astype(np.float32), std_out.astype(np.float32)


def train_rollout(net: UNet, snaps, steps: int, lr: float = 1e-3, seed: int = 0, log_every: int = 0,
                  pushforward: float = 0.5):
    """Adam on snapshot sequences [windows + 1, domains, ny, nx, 5]: a sample
    is a random (window w, domain d); with probability `pushforward` its input
    is the network's own prediction from window w and its target window
    w + 2, otherwise the input is window w and the target w + 1 (training on
    the network's own outputs keeps long rollouts close to the solver's
    states).  Cosine decay of the learning rate to a tenth.  Returns the loss
    history [(step, loss)] read every log_every steps."""
    import torch

    B = net.shape[0]
    n_w, n_d = int(snaps.shape[0]), int(snaps.shape[1])
    rng = np.random.Generator(np.random.PCG64(seed))
    xb = torch.empty(net.shape, dtype=torch.float32, device="cuda")
    tb = torch.empty_like(xb)
    yb = torch.empty_like(xb)
    hist = []
    for it in range(steps):
        pf = [bool(rng.random() < pushforward) and n_w >= 3 for _ in range(B)]
        for j in range(B):
            w = int(rng.integers(0, n_w - (2 if pf[j] else 1)))
            d = int(rng.integers(0, n_d))
            xb[j].copy_(snaps[w, d])
            tb[j].copy_(snaps[w + (2 if pf[j] else 1), d])
        if any(pf):
            net.forward(xb, yb)
            for j in range(B):
                if pf[j]:
                    xb[j].copy_(yb[j])
        a = lr * (0.1 + 0.9 * 0.5 * (1.0 + math.cos(math.pi * it / max(1, steps))))
        net.train_step(xb, tb, a)
        if log_every and (it % log_every == 0 or it == steps - 1):
            hist.append((it, net.loss()))
    return hist


def train(net: UNet, x, t, steps: int, lr: float = 1e-3, seed: int = 0, log_every: int = 0):
    """Adam on random mini-batches of (x, t) pairs (batch = the network's
    batch); cosine decay of the learning rate to a tenth.  Returns the loss
    history [(step, loss)] read every log_every steps."""
    import torch

    B = net.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    xb = torch.empty(net.shape, dtype=torch.float32, device="cuda")
    tb = torch.empty_like(xb)
    hist = []
    n = x.shape[0]
    for it in range(steps):
        idx = rng.integers(0, n, B)
        for j, i in enumerate(idx):  # device-to-device copies
            xb[j].copy_(x[int(i)])
            tb[j].copy_(t[int(i)])
        a = lr * (0.1 + 0.9 * 0.5 * (1.0 + math.cos(math.pi * it / max(1, steps))))
        net.train_step(xb, tb, a)
        if log_every and (it % log_every == 0 or it == steps - 1):
            hist.append((it, net.loss()))
    return hist


def rollout(sim, net: UNet, windows: int, K: int, tip_tol: float, audit_every: int, backoff: int,
            cx: float, cy: float, orient: float = 0.0, lb_first: int = 0, drift_budget: float | None = None,
            drift_factor: float = 1.0):
    """Surrogate-accelerated run of `windows` windows of K steps.

    Policy: the first lb_first windows are run by the plain LB; then the
    network advances windows, and every audit_every-th window is also run by
    the plain LB from the same state (the LB result is kept).  If the
    audit's tip error exceeds tip_tol, the state returns to the snapshot taken
    at the previous passed audit, every window since is re-run by the LB, and
    the network sits out the next `backoff` windows.  An unaudited window
    whose prediction is not finite is not applied and counts as a failed audit;
    so does a window in which the state or the audit's LB run goes non-finite
    (from a finite but unphysical prediction kept earlier).

    Drift budget: window errors add up over a rollout, which a one-window
    audit does not see.  Each passed audit charges drift_factor times its tip
    error for every network window it stands for (those since the previous
    audit); when the charges would exceed `drift_budget` (default tip_tol)
    with the next stretch, the network stops and the LB runs the remaining
    windows.
    Returns counts."""
    budget = tip_tol if drift_budget is None else drift_budget
    st = {"surrogate": 0, "audited": 0, "rejected": 0, "nonfinite": 0, "lb_rerun": 0, "lb_backoff": 0,
          "lb_first": 0, "lb_after_budget": 0, "drift_charged": 0.0, "tip_err": []}
    w = 0
    if lb_first:  # the first windows (fast early growth of the seed) by the LB
        n = min(lb_first, windows)
        sim.step(K * n)
        st["lb_first"] = n
        w = n
    sim.snapshot_save(0)
    since, off = 0, 0
    while w < windows:
        if off > 0:
            sim.step(K)
            st["lb_backoff"] += 1
            off -= 1
            w += 1
            if off == 0:
                sim.snapshot_save(0)
                since = 0
            continue
        audit = since + 1 >= audit_every or w == windows - 1
        try:
            rep = sim.surrogate_advance(net, K, tip_tol, audit, cx, cy, orient)
        except L.LBMError as err:
            # a finite but unphysical prediction kept in an earlier window can
            # make the state, or this window's LB audit, go non-finite: the
            # stretch since the last passed audit is rejected like a failed audit
            if err.code != L.LBM_ENUMERIC:
                raise
            rep = {"audited": audit, "accepted": False, "tip_err": math.inf, "nonfinite": True}
        w += 1
        if rep.get("nonfinite"):
            st["nonfinite"] += 1
        if not audit and rep["accepted"]:
            st["surrogate"] += 1
            since += 1
            continue
        if not audit:  # a prediction that is not finite was not applied: as a failed audit
            st["rejected"] += 1
            if not rep.get("nonfinite"):
                st["nonfinite"] += 1
            sim.snapshot_restore(0)
            sim.step(K * (since + 1))
            st["surrogate"] -= since
            st["lb_rerun"] += since
            off = backoff
            sim.snapshot_save(0)
            since = 0
            continue
        st["audited"] += 1
        st["tip_err"].append(rep["tip_err"])
        if rep["accepted"]:
            st["drift_charged"] += drift_factor * rep["tip_err"] * since
            sim.snapshot_save(0)
            since = 0
            if st["drift_charged"] + drift_factor * rep["tip_err"] * (audit_every - 1) > budget and w < windows:
                st["lb_after_budget"] = windows - w
                sim.step(K * (windows - w))
                w = windows
        else:
            st["rejected"] += 1
            st["surrogate"] -= since
            sim.snapshot_restore(0)
            sim.step(K * (since + 1))
            st["lb_rerun"] += since
            off = backoff
            sim.snapshot_save(0)
            since = 0
    return st


def _main(argv=None) -> int:
    """Command line: run the network forward (or one training step) on a
    seeded random field with seeded weights and print the device time;
    a target for profilers."""
    import argparse

    import torch

    from . import workloads

    ap = argparse.ArgumentParser(prog="python -m paper_2209_01444_gb300.surrogate")
    ap.add_argument("mode", choices=["forward", "train", "conv"])
    ap.add_argument("--size", type=int, default=1024)
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--cin", type=int, default=32, help="conv mode: input channels")
    ap.add_argument("--cout", type=int, default=32, help="conv mode: output channels")
    a = ap.parse_args(argv)
    if a.mode == "conv":
        return _conv_main(a)
    net = UNet(a.batch, a.size, a.size)
    net.set_params(workloads.unet_params(param_shapes(), 1))
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(a.batch, a.size, a.size, 5, generator=g, device="cuda")
    t = x + 0.01
    y = torch.empty_like(x)
    run = (lambda: net.forward(x, y)) if a.mode == "forward" else (lambda: net.train_step(x, t, 1e-4))
    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    print(f"{a.mode} batch {a.batch} {a.size}x{a.size}: {e0.elapsed_time(e1) / a.reps:.3f} ms per call")
    return 0


def _conv_main(a) -> int:
    """One implicit 3 x 3 convolution (lbm_nn_conv3x3) of a seeded field."""
    import torch

    lib = L.load()
    g = torch.Generator(device="cuda").manual_seed(0)
    X = torch.randn(a.batch, a.size, a.size, a.cin, generator=g, device="cuda").to(torch.bfloat16)
    Wm = (torch.randn(a.cout, 9 * a.cin, generator=g, device="cuda") * 0.05).to(torch.bfloat16)
    bias = torch.zeros(a.cout, device="cuda")
    D = torch.empty(a.batch * a.size * a.size, a.cout, dtype=torch.bfloat16, device="cuda")
    st = ct.c_void_p(torch.cuda.current_stream().cuda_stream)

    def run():
        rc = lib.lbm_nn_conv3x3(ct.c_void_p(X.data_ptr()), a.batch, a.size, a.size, a.cin, a.cin,
                                ct.c_void_p(Wm.data_ptr()), 9 * a.cin, ct.c_void_p(D.data_ptr()), a.cout,
                                ct.c_void_p(bias.data_ptr()), a.cout, 0, 1, st)
        if rc != L.LBM_OK:
            raise L.LBMError(rc, "lbm_nn_conv3x3")

    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    flop = 2.0 * a.batch * a.size * a.size * 9 * a.cin * a.cout
    print(f"conv {a.batch}x{a.size}x{a.size}, {a.cin} -> {a.cout}: {ms * 1e3:.1f} us, {flop / ms / 1e9:.0f} TFLOP/s")
    return 0


if __name__ == "__main__":
    raise SystemExit(_main())
