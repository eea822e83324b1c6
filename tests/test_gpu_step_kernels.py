"""The two kernels of the fused coupled step (register-staged tiled and
TMA-staged persistent) run the same per-node arithmetic, coupled_node, on the
same inputs; they differ in how the populations arrive.  Inlined into
different kernels, that arithmetic may still round differently where the
compiler fuses a product into a multiply-add, so the states must agree to
rounding: 1e-5 with FP32 storage after 37 steps.  With 16-bit storage one
rounding of a stored value may come out one step apart and spread for a few
steps: a deviation near 1-2 is stored as FP16 after a scale of 16 (step
2^-6 / 16 = 9.8e-4) or as BF16 unscaled (step 2^-7 = 7.8e-3), so 4e-3 and
2e-2.
A misplaced or missed load or store moves a population by O(0.1).  Every wall
type, ragged grids, grain maps and flow sub-steps; also the kernel choice."""
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


def _both(L, p, start, steps, storage="fp32"):
    out = []
    for kernel in ("tma", "tiled"):
        s = L.Simulation(p, storage)
        s.set_step_kernel(kernel)
        assert s.step_kernel == kernel
        start(s)
        s.step(steps)
        s.synchronize()
        out.append(s.state())
    return out


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("shape", [(48, 10), (70, 45), (129, 67)])
@pytest.mark.parametrize("bcs", sorted(BCS))
def test_tma_kernel_equals_tiled_kernel(lbm, bcs, shape, storage):
    """Random fields with four grains; ragged tiles in x and y, and the
    smallest grid the 16-bit TMA kernel takes (one phi box wide)."""
    nx, ny = shape
    p = W.thermosolutal_params(nx, ny, bc=BCS[bcs], u_in=(0.15, 0.02), gbetaT=W.GBETA_T * 5,
                               gbetaC=W.GBETA_C * 5, theta_ref=-0.5, dir_theta=-0.4)
    f, orient = W.random_fields(nx, ny, rng_seed=3 + nx)
    a, b = _both(lbm, p, lambda s: s.init_fields(f, orient), 37, storage)
    _agree(a, b, storage)


def test_tma_kernel_smallest_fp32_grid(lbm):
    p = W.thermosolutal_params(40, 10, bc=BCS["mixed"], u_in=(0.15, 0.02), gbetaT=W.GBETA_T * 5)
    f, orient = W.random_fields(40, 10, rng_seed=43)
    a, b = _both(lbm, p, lambda s: s.init_fields(f, orient), 37)
    _agree(a, b, "fp32")


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("n_sub", [1, 3])
def test_tma_kernel_equals_tiled_kernel_seeded(lbm, n_sub, storage):
    """Multi-seed start with a grain map on 256 x 192, and the flow sub-steps
    (the kernel then also writes the frozen force plane)."""
    c = W.multi_seed(n=256, count=6, min_spacing=60.0)
    p = dict(c.params, ny=192, n_sub=n_sub, nu=2.0 * n_sub)
    seeds = c.seeds[c.seeds[:, 1] < 180]
    a, b = _both(lbm, p, lambda s: s.init_seeds(seeds, c.U0, c.theta0), 50, storage)
    _agree(a, b, storage)


def test_kernel_choice(lbm):
    big = W.thermosolutal_params(64, 64)
    s = lbm.Simulation(big)
    assert s.step_kernel == "tiled"         # the default
    s.set_step_kernel("tma")
    assert s.step_kernel == "tma"
    s.set_step_kernel("auto")
    assert s.step_kernel == "tiled"
    s.set_step_kernel("tma")
    small = lbm.Simulation(W.thermosolutal_params(39, 64))
    assert small.step_kernel == "tiled"     # narrower than one f box
    with pytest.raises(lbm.LBMError):
        small.set_step_kernel("tma")
    h = lbm.Simulation(big, "fp16")
    assert h.step_kernel == "tiled"
    h.set_step_kernel("tma")
    assert h.step_kernel == "tma"
    with pytest.raises(lbm.LBMError):       # 16-bit: the phi box is 48 wide
        lbm.Simulation(W.thermosolutal_params(47, 64), "fp16").set_step_kernel("tma")
    assert s.lib.lbm_set_step_kernel(s.h, 7) < 0
    assert s.step_kernel == "tma"


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
