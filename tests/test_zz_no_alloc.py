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
