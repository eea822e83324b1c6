"""lbm_reduce_noalloc, the allocation-free reduction, against lbm_get_metrics.

Callers that cannot allocate device memory (their memory belongs to another
allocator, or they may only allocate at start-up) use lbm_reduce_noalloc on
population buffers they own; its scratch is a static device array of the
library.  This file is collected last so that a run stopping at the first
failure has run every other test before it.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np
import pytest

from paper_2209_01444_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _layout(params, storage):
    nx, ny = params["nx"], params["ny"]
    plane = (nx + 31) // 32 * 32 * ny
    sc = plane * (60 if storage == "fp32" else 36)
    fl = plane * (36 if storage == "fp32" else 18)
    # checkpoint: header, scalar buffer, flow buffer, 6 FP32 history planes,
    # grain ids, 256 (cos, sin) pairs
    tail = sc + fl + plane * 24 + plane + 256 * 8
    return sc, fl, tail


def _device_buffers(torch, sim, params, storage):
    """The state's scalar and flow buffers, copied from a checkpoint into
    device memory allocated by the test (torch), not by the library."""
    blob = sim.save()
    sc, fl, tail = _layout(params, storage)
    head = len(blob) - tail
    raw = np.frombuffer(blob, dtype=np.uint8)
    d_sc = torch.from_numpy(raw[head:head + sc].copy()).cuda()
    d_fl = torch.from_numpy(raw[head + sc:head + sc + fl].copy()).cuda()
    return d_sc, d_fl


def _noalloc(lbm, torch, params, storage, d_sc, d_fl, cx, cy, orient):
    lib = lbm.load()
    p = lbm.make_params(params, storage)
    out = torch.full((10,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = lib.lbm_reduce_noalloc(ct.byref(p), ct.c_void_p(d_sc.data_ptr()), ct.c_void_p(d_fl.data_ptr()), cx, cy,
                                orient, ct.c_void_p(out.data_ptr()), ct.c_void_p(stream.cuda_stream))
    assert rc == 0, lib.lbm_last_error(None)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _compare(got, m, nodes, vscale):
    assert got[0] / nodes == pytest.approx(m["solid_fraction"], rel=1e-12)
    for i, k in ((1, "sum_C"), (2, "sum_H"), (3, "sum_h"), (6, "sum_phi")):
        assert got[i] == pytest.approx(m[k], rel=1e-5, abs=1e-6), k
    assert got[4] / vscale == pytest.approx(m["max_u"], rel=1e-12)
    assert got[5] == 0 and m["nonfinite"] == 0
    for j, k in enumerate(("tip_px", "tip_mx", "tip_py")):
        assert got[7 + j] == pytest.approx(m[k], abs=1e-12), k


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_noalloc_reduction_matches_the_handle_reduction_twice_in_a_row(storage):
    torch = pytest.importorskip("torch")
    from paper_2209_01444_gb300 import build_ext, lbm

    build_ext.build()
    lbm.load()
    case = W.single_seed_periodic(n=128)
    sim = lbm.Simulation(case.params, storage, stream=torch.cuda.current_stream())
    sim.init_seeds(case.seeds, case.U0, case.theta0)
    vscale = case.params["dt"] / case.params["n_sub"] / case.params["dx"]
    for steps in (60, 90):            # two calls in a row, on two different states
        sim.step(steps)
        m = sim.metrics(64.0, 64.0, 0.2)
        d_sc, d_fl = _device_buffers(torch, sim, case.params, storage)
        got = _noalloc(lbm, torch, case.params, storage, d_sc, d_fl, 64.0, 64.0, 0.2)
        _compare(got, m, case.nodes, vscale)


def _exactly_equal(got, m, nodes, vscale):
    """Both paths fold the same per-node terms in the same blocks and order
    (one shared reduction routine), so every output is the same double."""
    assert got[0] / nodes == m["solid_fraction"]
    for i, k in ((1, "sum_C"), (2, "sum_H"), (3, "sum_h"), (6, "sum_phi")):
        assert got[i] == m[k], k
    assert got[4] / vscale == m["max_u"]
    assert got[5] == 0 and m["nonfinite"] == 0
    for j, k in enumerate(("tip_px", "tip_mx", "tip_py")):
        assert got[7 + j] == m[k], k


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_noalloc_reduction_on_a_ragged_grid_equals_the_handle_exactly(storage):
    """131 x 97 nodes: a row pitch of 160 (the padding columns must be
    skipped) and 12,707 nodes, so the last of the four blocks of 4096 nodes
    is partial (419 nodes).  Two calls in a row on two states, every output
    compared for equality."""
    torch = pytest.importorskip("torch")
    from paper_2209_01444_gb300 import build_ext, lbm

    build_ext.build()
    lbm.load()
    params = W.thermosolutal_params(131, 97, bc=("inflow", "outflow", "symmetry", "symmetry"), u_in=(0.2, 0.0),
                                    gbetaT=W.GBETA_T, gbetaC=W.GBETA_C)
    seeds = np.array([[49.0, 48.0, 7.0, 0.3]])
    sim = lbm.Simulation(params, storage, stream=torch.cuda.current_stream())
    sim.init_seeds(seeds, -0.2, -0.5)
    vscale = params["dt"] / params["n_sub"] / params["dx"]
    for steps in (25, 40):
        sim.step(steps)
        m = sim.metrics(49.0, 48.0, 0.3)
        d_sc, d_fl = _device_buffers(torch, sim, params, storage)
        got = _noalloc(lbm, torch, params, storage, d_sc, d_fl, 49.0, 48.0, 0.3)
        _exactly_equal(got, m, 131 * 97, vscale)


def test_noalloc_reduction_allocates_no_device_memory():
    """After one call (which looks up the static array's address), further
    calls change neither the device's free memory nor the memory the torch
    caching allocator holds: the entry point allocates nothing."""
    torch = pytest.importorskip("torch")
    from paper_2209_01444_gb300 import build_ext, lbm

    build_ext.build()
    lbm.load()
    case = W.single_seed_periodic(n=128)
    sim = lbm.Simulation(case.params, "fp32", stream=torch.cuda.current_stream())
    sim.init_seeds(case.seeds, case.U0, case.theta0)
    sim.step(10)
    d_sc, d_fl = _device_buffers(torch, sim, case.params, "fp32")
    first = _noalloc(lbm, torch, case.params, "fp32", d_sc, d_fl, 64.0, 64.0, 0.2)
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    lib = lbm.load()
    p = lbm.make_params(case.params, "fp32")
    out = torch.empty(10, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        rc = lib.lbm_reduce_noalloc(ct.byref(p), ct.c_void_p(d_sc.data_ptr()), ct.c_void_p(d_fl.data_ptr()), 64.0,
                                    64.0, 0.2, ct.c_void_p(out.data_ptr()), ct.c_void_p(stream.cuda_stream))
        assert rc == 0, lib.lbm_last_error(None)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0
    np.testing.assert_array_equal(out.cpu().numpy(), first)


_CAPTURE_FIRST = r"""
import ctypes as ct, sys
sys.path.insert(0, {root!r})
import torch
from paper_2209_01444_gb300 import lbm, workloads as W
lib = lbm.load()
p = lbm.make_params(W.thermosolutal_params(64, 64))
buf = torch.zeros(64 * 64 * 16, dtype=torch.float32, device="cuda")
out = torch.zeros(10, dtype=torch.float64, device="cuda")
torch.cuda.synchronize()
s = torch.cuda.Stream()
g = torch.cuda.CUDAGraph()
with torch.cuda.stream(s):
    g.capture_begin()
    rc = lib.lbm_reduce_noalloc(ct.byref(p), ct.c_void_p(buf.data_ptr()), ct.c_void_p(buf.data_ptr()), 0.0, 0.0,
                                0.0, ct.c_void_p(out.data_ptr()), ct.c_void_p(s.cuda_stream))
    msg = lib.lbm_last_error(None).decode()
    g.capture_end()
print(rc, msg)
"""


def test_noalloc_first_call_under_stream_capture_is_refused():
    """In a fresh process, a first call made while its stream is being
    captured has no device address of the static array yet (looking it up
    is not a stream operation): it is refused with LBM_EINVAL and a reason,
    and launches nothing."""
    pytest.importorskip("torch")
    import os
    import subprocess
    import sys

    from paper_2209_01444_gb300 import build_ext

    build_ext.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _CAPTURE_FIRST.format(root=root)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    rc, _, msg = r.stdout.strip().splitlines()[-1].partition(" ")
    assert int(rc) == -1 and "before capture" in msg, r.stdout


def test_noalloc_reduction_rejects_grids_beyond_its_limit():
    torch = pytest.importorskip("torch")
    from paper_2209_01444_gb300 import build_ext, lbm

    build_ext.build()
    lib = lbm.load()
    p = lbm.make_params(W.thermosolutal_params(8192, 4097))
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    rc = lib.lbm_reduce_noalloc(ct.byref(p), ct.c_void_p(dummy.data_ptr()), ct.c_void_p(dummy.data_ptr()), 0.0,
                                0.0, 0.0, ct.c_void_p(dummy.data_ptr()), None)
    assert rc == lbm.LBM_EINVAL
    assert b"33554432" in lib.lbm_last_error(None)
