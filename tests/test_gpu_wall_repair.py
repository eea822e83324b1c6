"""Inside the captured step graphs the left/right walls of one step are
updated by the next step as it loads them, instead of by the column pass of
the wall kernel.  The extrapolation depends on the interior node alone, so
the states must agree with direct launches (column pass after every step) to
rounding: the same arithmetic inlined into another kernel may fuse a product
into a multiply-add differently, 1e-5 with FP32 storage after 40 steps.  With
16-bit storage one rounding of a stored value may come out one step apart and
spread for a few steps: a deviation near 1-2 is stored as FP16 after a scale
of 16 (step 2^-6 / 16 = 9.8e-4), so 4e-3.  A misplaced or missed load or
store moves a population by O(0.1)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2209_01444_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp16": 4e-3, "bf16": 2e-2}


def _agree(a, b, storage):
    d = float(np.abs(a - b).max())
    print(f"{storage}: largest state difference {d:.2e}")
    assert d <= TOL[storage], d


@pytest.fixture(scope="module")
def lbm():
    from paper_2209_01444_gb300 import build_ext, lbm as L

    build_ext.build()
    L.load()
    return L


BCS = {
    "periodic": ("periodic",) * 4,
    "inflow_outflow_symmetry": ("inflow", "outflow", "symmetry", "symmetry"),
    "channel_noslip": ("periodic", "periodic", "noslip", "noslip"),
    "dirichlet": ("dirichlet",) * 4,
    "mixed": ("inflow", "outflow", "noslip", "symmetry"),
}


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("bcs", ["inflow_outflow_symmetry", "mixed", "dirichlet", "side_walls"])
def test_walls_repaired_at_load_match_the_column_pass(lbm, bcs, storage):
    """Inside the captured graphs the left/right walls of one step are updated
    by the next step as it loads them, instead of by the column pass.  The
    extrapolation depends on the interior node alone, so the states must agree
    with direct launches (column pass after every step) to rounding: the same
    arithmetic in another kernel.  40 steps = two graphs and a remainder; grids
    whose last tile holds only the right wall (nx - 1 = 64 or 32, the latter
    also in the previous tile's halo column), one without a right wall in
    its last tile's own columns (nx = 40), and one narrower than a tile (both
    walls in one tile)."""
    for nx, ny in ((65, 37), (29, 24), (40, 41), (33, 33)):
        bc = ("symmetry", "noslip", "periodic", "periodic") if bcs == "side_walls" else BCS[bcs]
        p = W.thermosolutal_params(nx, ny, bc=bc, u_in=(0.08, 0.01), gbetaT=W.GBETA_T * 5, dir_theta=-0.4)
        f, orient = W.random_fields(nx, ny, rng_seed=5 + nx)
        out = []
        for direct in (False, True):
            s = lbm.Simulation(p, storage)
            s.init_fields(f, orient)
            s.set_profiling(direct)  # direct launches only, column pass after each step
            s.step(40)
            s.synchronize()
            out.append(s.state())
        _agree(out[0], out[1], storage)
