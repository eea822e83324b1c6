"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Error metric per field X: max|X_gpu - X_ref| / max(max|X_ref|, floor_X) with
floors phi: 1, C: 1, U: 1, theta: |theta0|, u: 1e-6, p: 1e-6 (paper units).
Bound: 1e-4 for FP32 storage; 1e-2 (and tips within 1 lattice unit) for the
FP16/BF16 equilibrium-shifted storage.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import oracle as O
import storage_emulation as SE
from paper_2209_01444_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-4
LOWP_TOL = 1e-2
# FP32 rounding of the initial populations alone: the pressure is formed from
# populations whose velocity terms are up to 100x larger than it.
T0_TOL = 2e-5


@pytest.fixture(scope="module")
def lbm():
    import torch

    from paper_2209_01444_gb300 import build_ext, lbm as L

    build_ext.build()
    L.load()
    torch.cuda.init()
    return L


def floors(theta0=0.55):
    return {"phi": 1.0, "C": 1.0, "U": 1.0, "theta": abs(theta0), "ux": 1e-6, "uy": 1e-6, "p": 1e-6}


def field_errors(got, want, theta0=0.55):
    fl = floors(theta0)
    out = {}
    for k, v in want.items():
        scale = max(np.abs(v).max(), fl[k])
        out[k] = float(np.abs(got[k] - v).max() / scale)
    return out


def assert_close(got, want, tol, theta0=0.55, where=""):
    errs = field_errors(got, want, theta0)
    bad = {k: e for k, e in errs.items() if not e <= tol}
    assert not bad, f"{where}: {bad} (all: {errs})"


class Checkpoints:
    """Collect the errors of every checkpoint, fail once at the end with all."""

    def __init__(self):
        self.rows, self.bad = [], []

    def add(self, got, want, tol, theta0, where):
        errs = field_errors(got, want, theta0)
        self.rows.append((where, errs))
        if any(not e <= tol for e in errs.values()):
            self.bad.append(where)

    def check(self):
        table = "\n".join(f"{w}: " + ", ".join(f"{k}={v:.2e}" for k, v in e.items()) for w, e in self.rows)
        assert not self.bad, f"failed at {self.bad}\n{table}"


def pair(lbm, params, storage="fp32"):
    return lbm.Simulation(params, storage), O.Oracle(params)


# ------------------------------------------------------------------ starts
def test_seeded_start_matches(lbm):
    c = W.single_seed_periodic()
    g, o = pair(lbm, c.params)
    g.init_seeds(c.seeds, c.U0, c.theta0)
    o.init_seeds(c.seeds, c.U0, c.theta0)
    assert_close(g.fields(), o.fields(), T0_TOL, where="t=0")
    np.testing.assert_allclose(g.state(), o.state(), rtol=0, atol=1e-6)


def test_multi_seed_grain_map_and_start(lbm):
    c = W.multi_seed(n=256, count=6, min_spacing=60.0)
    g, o = pair(lbm, c.params)
    g.init_seeds(c.seeds, c.U0, c.theta0)
    o.init_seeds(c.seeds, c.U0, c.theta0)
    assert_close(g.fields(), o.fields(), T0_TOL, c.theta0, where="t=0")
    g.step(30)
    o.step(30)
    assert_close(g.fields(), o.fields(), FP32_TOL, c.theta0, where="t=30")


# ------------------------------------------------------------------ runs
def test_single_seed_periodic_box_1000_steps(lbm):
    """128 x 128 periodic box, one seed R = 8, Delta = 0.55, eps = 0.05,
    buoyancy on: fields match the oracle at steps 1, 10, 100 and 1000."""
    c = W.single_seed_periodic()
    g, o = pair(lbm, c.params)
    g.init_seeds(c.seeds, c.U0, c.theta0)
    o.init_seeds(c.seeds, c.U0, c.theta0)
    cp = Checkpoints()
    for T in (1, 10, 100, 1000):
        g.step(T - g.steps)
        o.step(T - o.steps)
        cp.add(g.fields(), o.fields(), FP32_TOL, 0.55, f"step {T}")
    cp.check()


BCS = {
    "periodic": ("periodic",) * 4,
    "inflow_outflow_symmetry": ("inflow", "outflow", "symmetry", "symmetry"),
    "channel_noslip": ("periodic", "periodic", "noslip", "noslip"),
    "dirichlet": ("dirichlet",) * 4,
    "mixed": ("inflow", "outflow", "noslip", "symmetry"),
}


@pytest.mark.parametrize("shape", [(37, 23), (70, 45)])
@pytest.mark.parametrize("bcs", sorted(BCS))
def test_random_fields_parity(lbm, bcs, shape):
    """Random smooth fields (liquid, solid and interface, flow, four grains)
    on grids spanning several tiles with ragged tails, every wall type."""
    nx, ny = shape
    p = W.thermosolutal_params(nx, ny, bc=BCS[bcs], u_in=(0.15, 0.02), gbetaT=W.GBETA_T * 5,
                               gbetaC=W.GBETA_C * 5, theta_ref=-0.5, dir_theta=-0.4)
    f, orient = W.random_fields(nx, ny, rng_seed=11 + nx)
    if bcs == "dirichlet":
        # as in the far-field runs of Sec. 4.4, the walls start at the imposed
        # values (a start that violates them switches phi by O(1) in one step
        # where grad(phi) is tiny, which makes the direction of J_at, Eq. (7),
        # a matter of rounding)
        for q, v in ((0, -1.0), (1, 0.0), (2, -0.4)):
            f[q][0, :] = f[q][-1, :] = v
            f[q][:, 0] = f[q][:, -1] = v
    g, o = pair(lbm, p)
    g.init_fields(f, orient)
    o.init_fields(f, orient)
    cp = Checkpoints()
    cp.add(g.fields(), o.fields(), T0_TOL, 0.5, "t=0")
    for T in (1, 5, 60):
        g.step(T - g.steps)
        o.step(T - o.steps)
        cp.add(g.fields(), o.fields(), FP32_TOL, 0.5, f"{bcs} {shape} step {T}")
    cp.check()


@pytest.mark.parametrize("shape,bcs", [((4, 4), "periodic"), ((4, 6), "channel_noslip"),
                                       ((5, 4), "inflow_outflow_symmetry"), ((32, 5), "mixed"),
                                       ((33, 4), "periodic"), ((31, 7), "channel_noslip")])
def test_smallest_and_block_edge_grids_match_the_oracle(lbm, shape, bcs):
    """The smallest grid the library accepts (4 x 4), grids narrower and
    shorter than one tile (the tile's own cells and halo wrap onto the same
    few nodes), and row widths of 31, 32 and 33 nodes (one node-block of 32
    along x, and one node into a second): random fields against the oracle."""
    nx, ny = shape
    p = W.thermosolutal_params(nx, ny, bc=BCS[bcs], u_in=(0.15, 0.02), gbetaT=W.GBETA_T * 5,
                               gbetaC=W.GBETA_C * 5, theta_ref=-0.5, dir_theta=-0.4)
    f, orient = W.random_fields(nx, ny, rng_seed=3 + nx * ny)
    g, o = pair(lbm, p)
    g.init_fields(f, orient)
    o.init_fields(f, orient)
    cp = Checkpoints()
    for T in (1, 5, 30):
        g.step(T - g.steps)
        o.step(T - o.steps)
        cp.add(g.fields(), o.fields(), FP32_TOL, 0.5, f"{bcs} {shape} step {T}")
    cp.check()


def test_tallest_grid_matches_the_oracle(lbm):
    """The tallest grid the library accepts (ny = 262140: the launches of
    64 x 4-node blocks reach the 65535 limit of the grid's y dimension),
    about a million nodes: random fields against the oracle over three steps."""
    nx, ny = 4, 262140
    p = W.thermosolutal_params(nx, ny, bc=BCS["channel_noslip"], u_in=(0.15, 0.02), gbetaT=W.GBETA_T * 5,
                               gbetaC=W.GBETA_C * 5, theta_ref=-0.5, dir_theta=-0.4)
    f, orient = W.random_fields(nx, ny, rng_seed=7)
    g, o = pair(lbm, p)
    g.init_fields(f, orient)
    o.init_fields(f, orient)
    cp = Checkpoints()
    for T in (1, 3):
        g.step(T - g.steps)
        o.step(T - o.steps)
        cp.add(g.fields(), o.fields(), FP32_TOL, 0.5, f"(4, 262140) step {T}")
    cp.check()


def test_widest_tested_grid_matches_the_oracle(lbm):
    """A strip 65543 nodes wide and 16 high (2049 node blocks per row, the
    last holding 7 nodes; about a million nodes) with inflow, outflow and
    no-slip walls, 40 seeds of radius 3-5 along it: against the oracle over
    three steps.  (Random fields, whose phi jumps between -1 and +1 from one
    row to the next, are not used on such strips: there the gradient of a flat
    wall row lies within FP32 rounding of the degenerate threshold at some
    nodes, and the jump of a_s it switches is pushed into the one-node spike
    next to it, an O(1e-2) difference between two admissible results.)"""
    nx, ny = 65543, 16
    p = W.thermosolutal_params(nx, ny, bc=BCS["mixed"], u_in=(0.05, 0.0), gbetaT=W.GBETA_T * 5,
                               gbetaC=W.GBETA_C * 5)
    r = np.random.Generator(np.random.PCG64(21))
    seeds = np.stack([np.linspace(800.0, nx - 800.0, 40), r.uniform(6.0, 9.0, 40), r.uniform(3.0, 5.0, 40),
                      r.uniform(0.0, math.pi / 4, 40)], axis=1)
    g, o = pair(lbm, p)
    g.init_seeds(seeds, -0.2, -0.45)
    o.init_seeds(seeds, -0.2, -0.45)
    cp = Checkpoints()
    for T in (1, 3):
        g.step(T - g.steps)
        o.step(T - o.steps)
        cp.add(g.fields(), o.fields(), FP32_TOL, 0.45, f"(65543, 16) step {T}")
    cp.check()


def _uniform(nx, ny, phi, U, theta, ux=0.0, uy=0.0):
    f = np.zeros((6, ny, nx))
    f[0], f[1], f[2], f[3], f[4] = phi, U, theta, ux, uy
    return f


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("state", ["undercooled_melt", "solid", "melt_in_uniform_flow"])
def test_uniform_states_stay_uniform_and_match_the_oracle(lbm, state, storage):
    """Degenerate states of the method on a periodic grid: with no interface
    grad(phi) = 0 at every node (the anisotropy's normal is undefined and the
    degenerate-gradient branch is taken everywhere); phi = -1 and +1 are fixed
    points of the phase-field equation, whose source has the factor 1 - phi^2.
    Every node computes the same arithmetic on the same values, so the fields
    must stay exactly uniform (a bit-exact invariant of the GPU path); the
    values must match the oracle, and phi must stay at +-1 to the rounding of
    its stored populations."""
    nx, ny = 40, 36
    p = W.thermosolutal_params(nx, ny, bc=BCS["periodic"], gbetaT=W.GBETA_T * 5, gbetaC=W.GBETA_C * 5,
                               theta_ref=-0.5)
    phi = 1.0 if state == "solid" else -1.0
    ux, uy = (0.05, -0.02) if state == "melt_in_uniform_flow" else (0.0, 0.0)
    f = _uniform(nx, ny, phi, -0.2, -0.45, ux, uy)
    g, o = lbm.Simulation(p, storage), O.Oracle(p)
    g.init_fields(f)
    o.init_fields(f)
    for T in (1, 50):
        g.step(T - g.steps)
        o.step(T - o.steps)
        got, want = g.fields(), o.fields()
        for k, v in got.items():
            assert v.max() == v.min(), (state, storage, T, k, float(v.max() - v.min()))
        assert np.abs(got["phi"] - phi).max() <= (1e-6 if storage == "fp32" else 1e-3)
        # the pressure of these states is 1e-7 .. 1e-4, formed from flow
        # populations of order 0.1 - 1: FP32 rounding of those alone moves it by
        # a few 1e-8, so it is compared in absolute terms.  With 16-bit storage
        # the bar applies to the transported fields and the velocity, as in the
        # other 16-bit tests (the rounding of the stored flow deviations moves p
        # by up to 4e-5 here, the same at every node)
        p_got, p_want = got.pop("p"), want.pop("p")
        if storage == "fp32":
            assert np.abs(p_got - p_want).max() <= 1e-6, (state, T, float(np.abs(p_got - p_want).max()))
        assert_close(got, want, FP32_TOL if storage == "fp32" else LOWP_TOL, -0.45, f"{state} {storage} step {T}")


@pytest.mark.parametrize("n_sub,h_kind", [(3, 0), (1, 1), (4, 1)])
def test_flow_substeps_and_h_kind(lbm, n_sub, h_kind):
    nx, ny = 48, 40
    p = W.thermosolutal_params(nx, ny, bc=BCS["inflow_outflow_symmetry"], u_in=(0.3, 0.0), n_sub=n_sub,
                               h_kind=h_kind, nu=2.0 * n_sub, gbetaT=W.GBETA_T, theta_ref=-0.5)
    f, orient = W.random_fields(nx, ny, rng_seed=5)
    g, o = pair(lbm, p)
    g.init_fields(f, orient)
    o.init_fields(f, orient)
    cp = Checkpoints()
    for T in (1, 40):
        g.step(T - g.steps)
        o.step(T - o.steps)
        cp.add(g.fields(), o.fields(), FP32_TOL, 0.5, f"n_sub={n_sub} h={h_kind} step {T}")
    cp.check()


@pytest.mark.parametrize("storage,bcs", [("fp32", "mixed"), ("fp32", "dirichlet"), ("fp32", "channel_noslip"),
                                         ("fp16", "mixed"), ("fp16", "channel_noslip")])
def test_flow_substeps_every_wall_type(lbm, bcs, storage):
    """Flow sub-steps on every wall type, corners included: between sub-steps
    the wall nodes are updated as the next sub-step loads them (rows from
    their interior node, columns from theirs, a corner from the row node beside
    it, each value rounded as the storage would round it), and the last
    sub-step of each coupled step runs the full wall pass.  FP32 within the
    FP32 bound, FP16 storage within the 16-bit bound.  FP16 with Dirichlet
    walls is checked from a seeded start below: from this random start it has
    a transient at steps 2-3 that does not involve the flow walls (the same at
    n_sub = 1; see test_reduced_precision_with_dirichlet_walls)."""
    nx, ny = 45, 38
    p = W.thermosolutal_params(nx, ny, bc=BCS[bcs], u_in=(0.2, 0.03), n_sub=3, nu=6.0, gbetaT=W.GBETA_T * 5,
                               theta_ref=-0.5, dir_theta=-0.4)
    f, orient = W.random_fields(nx, ny, rng_seed=21)
    g, o = pair(lbm, p, storage)
    g.init_fields(f, orient)
    o.init_fields(f, orient)
    cp = Checkpoints()
    # 16-bit storage: the bar applies to the transported fields and the
    # velocity (U multiplies C errors by up to 16 in the solid, and p is a
    # small difference of large populations)
    keep = None if storage == "fp32" else ("phi", "C", "theta", "ux", "uy")
    tol = FP32_TOL if storage == "fp32" else LOWP_TOL
    for T in (1, 2, 30):
        g.step(T - g.steps)
        o.step(T - o.steps)
        got, want = g.fields(), o.fields()
        if keep:
            got, want = {k: got[k] for k in keep}, {k: want[k] for k in keep}
        cp.add(got, want, tol, 0.5, f"{bcs} n_sub=3 {storage} step {T}")
    cp.check()


def test_reduced_precision_with_dirichlet_walls(lbm):
    """FP16 storage with Dirichlet walls on all sides (the far field of Sec.
    4.4) from a seeded start: within the 16-bit bound at every checkpoint.
    (From a random start whose phi meets the wall's value within one node, FP16
    shows a transient of up to 3e-2 at steps 2-3 next to the walls, down to
    2e-3 by step 5; periodic walls from the same start and FP32 storage show
    none.  The oracle with the same 16-bit rounding of its state shows it too:
    test_fp16_storage_matches_the_oracle_with_fp16_storage.)"""
    nx, ny = 45, 38
    p = W.thermosolutal_params(nx, ny, bc=BCS["dirichlet"], dir_theta=-0.5, theta_ref=-0.5)
    seeds = np.array([[22.0, 19.0, 6.0, 0.3]])
    g, o = pair(lbm, p, "fp16")
    g.init_seeds(seeds, -0.3, -0.5)
    o.init_seeds(seeds, -0.3, -0.5)
    cp = Checkpoints()
    for T in (1, 2, 3, 5, 30):
        g.step(T - g.steps)
        o.step(T - o.steps)
        got, want = g.fields(), o.fields()
        keep = ("phi", "C", "theta")
        cp.add({k: got[k] for k in keep}, {k: want[k] for k in keep}, LOWP_TOL, 0.5, f"dirichlet fp16 step {T}")
    cp.check()


@pytest.mark.parametrize("bcs", ["dirichlet", "periodic"])
def test_fp16_storage_matches_the_oracle_with_fp16_storage(lbm, bcs):
    """The FP16 path against the FP64 oracle whose state is rounded as the
    FP16 storage rounds it after every step: the two agree far below the
    16-bit error itself.  The Dirichlet case from this random start is where
    FP16 storage departs most from the unrounded oracle (3e-2 at step 2, next
    to the walls); the rounded oracle shows the same departure, so it is a
    property of 16-bit storage of this state, not of the kernels."""
    nx, ny = 45, 38
    p = W.thermosolutal_params(nx, ny, bc=BCS[bcs], u_in=(0.2, 0.03), gbetaT=W.GBETA_T * 5, theta_ref=-0.5,
                               dir_theta=-0.4)
    f, orient = W.random_fields(nx, ny, rng_seed=21)
    g = lbm.Simulation(p, "fp16")
    o, r = O.Oracle(p), O.Oracle(p)
    g.init_fields(f, orient)
    o.init_fields(f, orient)
    r.init_fields(f, orient)
    SE.round_state(r, p, "fp16")
    keep = ("phi", "C", "theta")
    for T in range(1, 6):
        g.step(1)
        o.step(1)
        r.step(1)
        SE.round_state(r, p, "fp16")
        G, Ro, Rr = g.fields(), o.fields(), r.fields()
        vs_rounded = field_errors({k: G[k] for k in keep}, {k: Rr[k] for k in keep})
        vs_plain = field_errors({k: G[k] for k in keep}, {k: Ro[k] for k in keep})
        print(bcs, T, {k: f"{vs_rounded[k]:.1e} / {vs_plain[k]:.1e}" for k in keep})
        assert max(vs_rounded.values()) <= 2e-3, (T, vs_rounded, vs_plain)


def test_metrics_match(lbm):
    c = W.single_seed_periodic()
    g, o = pair(lbm, c.params)
    g.init_seeds(c.seeds, c.U0, c.theta0)
    o.init_seeds(c.seeds, c.U0, c.theta0)
    g.step(300)
    o.step(300)
    for orient in (0.0, 0.35):
        mg, mo = g.metrics(64, 64, orient), o.metrics(64, 64, orient)
        for k in ("tip_px", "tip_mx", "tip_py"):
            assert mg[k] == pytest.approx(mo[k], abs=2e-3), k
        for k in ("solid_fraction", "sum_C", "sum_H", "sum_h", "sum_phi"):
            assert mg[k] == pytest.approx(mo[k], rel=1e-5, abs=1e-6), k
        assert mg["max_u"] == pytest.approx(mo["max_u"], rel=1e-3)
        assert mg["nonfinite"] == 0 and mg["step"] == 300


# ------------------------------------------------------------------ state
def test_graph_replay_equals_direct_launches(lbm):
    c = W.single_seed_periodic(n=64, R=6.0)
    a = lbm.Simulation(c.params)
    b = lbm.Simulation(c.params)
    for s in (a, b):
        s.init_seeds(c.seeds, c.U0, c.theta0)
    a.step(37)          # two captured 16-step graphs + 5 direct steps
    for _ in range(37):
        b.step(1)
    np.testing.assert_array_equal(a.state(), b.state())


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_checkpoint_resume_is_bit_exact(lbm, storage):
    c = W.single_seed_periodic(n=64, R=6.0)
    a = lbm.Simulation(c.params, storage)
    a.init_seeds(c.seeds, c.U0, c.theta0)
    a.step(20)
    blob = a.save()
    a.step(25)
    b = lbm.Simulation(c.params, storage)
    b.load(blob)
    assert b.steps == 20
    b.step(25)
    np.testing.assert_array_equal(a.state(), b.state())


def test_state_round_trip(lbm):
    p = W.thermosolutal_params(40, 30)
    f, orient = W.random_fields(40, 30, rng_seed=2)
    g = lbm.Simulation(p)
    g.init_fields(f, orient)
    g.step(3)
    st = g.state()
    g.set_state(st)
    np.testing.assert_allclose(g.state(), st, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(g.state_region(5, 7, 20, 11), g.state()[:, 7:18, 5:25])


def test_non_finite_state_is_reported(lbm):
    """Non-finite values are refused on the host by lbm_set_state; populations
    large enough to overflow FP32 sums are caught by the FP64 reduction and
    reported as LBM_ENUMERIC (no device fault involved)."""
    p = W.thermosolutal_params(32, 32)
    g = lbm.Simulation(p)
    f, orient = W.random_fields(32, 32, rng_seed=4)
    g.init_fields(f, orient)
    st = g.state()
    bad = st.copy()
    bad[0, 10, 10] = np.inf
    with pytest.raises(lbm.LBMError) as e:
        g.set_state(bad)
    assert e.value.code == lbm.LBM_EINVAL
    assert g.metrics(16, 16)["nonfinite"] == 0
    big = st.copy()
    big[0:5, 10, 10] = 3.0e38      # finite in FP32, their sum is not
    g.set_state(big)
    m = g.metrics(16, 16, check=False)
    assert m["rc"] == lbm.LBM_ENUMERIC and m["nonfinite"] == 1


# ------------------------------------------------------------------ precision
@pytest.mark.parametrize("storage,steps", [("fp16", 1000), ("bf16", 20)])
def test_reduced_precision_storage_accuracy(lbm, storage, steps):
    """Equilibrium-shifted 16-bit population storage with FP32 collisions: the
    transported fields within 1e-2 of the FP64 oracle and the tips within one
    lattice unit.  FP16 holds this for the whole 1000-step run; BF16 (8-bit
    mantissa) holds it for tens of steps only, after which the solute error
    grows until the run diverges (measured), so it is checked over 20 steps."""
    c = W.single_seed_periodic()
    g = lbm.Simulation(c.params, storage)
    o = O.Oracle(c.params)
    g.init_seeds(c.seeds, c.U0, c.theta0)
    o.init_seeds(c.seeds, c.U0, c.theta0)
    g.step(steps)
    o.step(steps)
    errs = field_errors(g.fields(), o.fields())
    mg, mo = g.metrics(64, 64), o.metrics(64, 64)
    tips = {k: (mg[k], mo[k]) for k in ("tip_px", "tip_mx", "tip_py")}
    # U (Eq. 20) is derived from C and phi and multiplies C errors by up to
    # 2/(k(1-k)) ~ 16 in the solid; the bar applies to the transported fields
    assert max(errs["phi"], errs["C"], errs["theta"]) <= LOWP_TOL, (errs, tips)
    for k, (a, b) in tips.items():
        assert abs(a - b) <= 1.0, (k, a, b, errs)
