"""Pins of the oracle's flow-only steps and hydrodynamic force (Eq. 27):
momentum balance of a body-force-driven periodic array of discs, the mirror
symmetry of that flow, and frozen scalar fields."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O
from paper_2209_01444_gb300 import workloads as W


def _periodic_disc(n=40, R=6.0, g=1e-5, nu=0.5):
    # dx = dt = 1: paper units are lattice units; the force is a body force per node
    p = W.thermosolutal_params(n, n, dx=1.0, dt=1.0, nu=nu, force=(g, 0.0), D=0.5, alpha=0.5)
    o = O.Oracle(p)
    o.init_seeds(np.array([[n / 2, n / 2, R, 0.0]]), 0.0, -0.55)
    return o, p


def test_force_balances_body_force_at_steady_state():
    """Periodic domain: each step changes the total momentum by the body force
    on every node plus the fluid-solid force, so at steady state the force on
    the solid equals N g."""
    n, g = 40, 1e-5
    o, _ = _periodic_disc(n=n, g=g)
    o.step_flow(3000)
    f1 = o.force(n / 2, n / 2)
    o.step_flow(1000)
    f2 = o.force(n / 2, n / 2)
    assert abs(f2[0] - f1[0]) <= 1e-4 * abs(f2[0]), "not steady"
    assert abs(f2[0] - n * n * g) <= 2e-4 * n * n * g, (f2[0], n * n * g)
    # mirror symmetry about the disc's horizontal axis: no lift, and no torque
    # apart from the row y = 0, its own mirror image under the periodic wrap,
    # where the diffuse solid weight is ~1e-5
    assert abs(f2[1]) <= 1e-9 * abs(f2[0])
    assert abs(f2[2]) <= 1e-6 * abs(f2[0]) * n


def test_flow_only_steps_freeze_scalars():
    o, _ = _periodic_disc()
    a = o.fields()
    o.step_flow(50)
    b = o.fields()
    for k in ("phi", "C", "U", "theta"):
        np.testing.assert_array_equal(a[k], b[k])
    assert np.abs(b["ux"]).max() > 0.0
    assert o.steps == 0


def test_force_sign_and_solid_share():
    """A uniform momentum in a fully solid box is pushed back: f = -u* at
    every node with weight 1, so F_f = +N u* along the flow."""
    n = 12
    p = W.thermosolutal_params(n, n, dx=1.0, dt=1.0, nu=0.5, D=0.5, alpha=0.5)
    o = O.Oracle(p)
    phi = np.ones((n, n))
    u = 0.01
    fields = np.stack([phi, np.zeros_like(phi), np.full_like(phi, -0.55), np.full_like(phi, u),
                       np.zeros_like(phi), np.zeros_like(phi)])
    o.init_fields(fields)
    fx, fy, _ = o.force(n / 2, n / 2)
    # the equilibrium start carries momentum u, so u* = u and f = -u everywhere
    assert abs(fx - n * n * u) <= 1e-12 and abs(fy) <= 1e-15
