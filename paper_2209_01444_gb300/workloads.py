"""Seeded synthetic inputs: parameter sets, seed layouts and random fields.

This module is the only thing the CUDA path and the FP64 oracle have in
common.  It holds no arithmetic of the method itself: it produces the problem
statement (the parameters in the paper's W0/tau0 units, seed positions and
radii, random initial fields) from a named configuration and an RNG seed, and
both sides turn that statement into populations with their own code.

Random numbers come from ``numpy.random.Generator(PCG64(seed))``.

Parameter dictionaries carry the fields of the paper's problem statement
(Secs. 2-4): ``nx, ny, W0, tau0, dx, dt, eps_s, lambda_, k, Mc_inf, D, alpha,
nu, rho0, n_sub, h_kind, gbetaT, gbetaC, theta_ref, C_ref, force, bc, u_in,
dir_phi, dir_U, dir_theta``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Lattice spacing and time step of every configuration below, in the paper's
# units: dx = W0, dt = tau0/20, so W0^2/tau0 = 0.05 lattice units, the thermal
# lattice diffusivity unit of the paper's Sec. 4.2 run (0.008/0.4^2).
DX = 1.0
DT = 0.05


def thermosolutal_params(nx: int, ny: int, **over) -> dict:
    """The thermosolutal parameter set of Sec. 4.4 (alpha = D = 2, k = 0.15,
    Mc_inf = 0.5325, lambda = 3.1913) with W0 = tau0 = 1, dx = 1, dt = 0.05,
    nu = 2 (lattice viscosity 0.1, Pr = 1), rho0 = 1, periodic walls, no
    forces."""
    p = dict(nx=nx, ny=ny, W0=1.0, tau0=1.0, dx=DX, dt=DT,
             eps_s=0.05, lambda_=3.1913, k=0.15, Mc_inf=0.5325,
             D=2.0, alpha=2.0, nu=2.0, rho0=1.0, n_sub=1, h_kind=0,
             gbetaT=0.0, gbetaC=0.0, theta_ref=-0.55, C_ref=1.0,
             force=(0.0, 0.0), bc=("periodic",) * 4, u_in=(0.0, 0.0),
             dir_phi=-1.0, dir_U=0.0, dir_theta=-0.55, grad_mode=0, isothermal=0)
    p.update(over)
    return p


def thermal_params(nx: int, ny: int, **over) -> dict:
    """The thermal (pure substance) set of Sec. 4.2: dx = 0.4 W0,
    dt = 0.008 tau0, eps = 0.05, Mc_inf = 0, alpha = 4, d0 = 0.1385 W0,
    lambda = a1 W0/d0 with a1 = 0.8839, symmetry walls."""
    lam = 0.8839 / 0.1385
    p = thermosolutal_params(nx, ny, dx=0.4, dt=0.008, eps_s=0.05, Mc_inf=0.0, alpha=4.0, D=4.0,
                             lambda_=lam, nu=4.0 * 23.1, bc=("symmetry",) * 4, theta_ref=-0.55)
    p.update(over)
    return p


def solutal_params(n: int, flow: bool = False, **over) -> dict:
    """The isothermal alloy of Sec. 4.3: L = n dx with dx = 0.4 W0 (as in
    Sec. 4.2), dt = 0.02 tau0, eps = 0.02, theta0 = 0 with no latent heat,
    D = 2, Mc_inf = 1, k = 0.15, lambda = 3.191 (d0 = a1 W0/lambda = 0.277 W0),
    symmetry walls.  With flow: inflow of 1 W0/tau0 on the left, outflow on
    the right, and the viscosity and n_sub = 15 of the Sec. 4.2 flow run (the
    paper gives neither for this case)."""
    p = thermosolutal_params(n, n, dx=0.4, dt=0.02, eps_s=0.02, Mc_inf=1.0, alpha=2.0, D=2.0, k=0.15,
                             lambda_=3.191, nu=4.0 * 23.1, bc=("symmetry",) * 4, theta_ref=0.0,
                             dir_theta=0.0, isothermal=1)
    if flow:
        p.update(n_sub=15, bc=("inflow", "outflow", "symmetry", "symmetry"), u_in=(1.0, 0.0))
    p.update(over)
    return p


# Buoyancy coefficients of the thermosolutal configurations: 1e-5 per unit
# theta (and -1e-5 per unit C) in lattice force units, i.e. 1e-5 * dx/dt^2 in
# paper units.
GBETA_T = 1e-5 * DX / DT**2
GBETA_C = -1e-5 * DX / DT**2


@dataclass
class Case:
    """One simulation: its parameters, seeds [x, y, R, orientation] in lattice
    units/radians, initial supersaturation U0 and temperature theta0, and the
    number of coupled steps."""
    name: str
    params: dict
    seeds: np.ndarray
    U0: float
    theta0: float
    steps: int
    meta: dict = field(default_factory=dict)

    @property
    def nodes(self) -> int:
        return int(self.params["nx"]) * int(self.params["ny"])


def single_seed_periodic(n: int = 128, steps: int = 1000, R: float = 8.0, **over) -> Case:
    """128 x 128 periodic box, one seed of radius 8 at the centre, Delta = 0.55,
    eps = 0.05, uniform U0 = 0, fluid at rest, thermal and solutal buoyancy."""
    p = thermosolutal_params(n, n, eps_s=0.05, gbetaT=GBETA_T, gbetaC=GBETA_C, theta_ref=-0.55)
    p.update(over)
    seeds = np.array([[n / 2, n / 2, R, 0.0]])
    return Case(f"single_seed_periodic_{n}", p, seeds, 0.0, -0.55, steps)


def forced_flow(n: int = 1024, steps: int = 20000, u_lattice: float = 0.01, **over) -> Case:
    """One seed of radius 10 at (3n/8, n/2) in a melt entering on the left at
    u_x = 0.01 (lattice units) and leaving on the right, symmetry walls at the
    top and bottom; Delta = 0.55, eps = 0.05, no buoyancy."""
    p = thermosolutal_params(n, n, eps_s=0.05, bc=("inflow", "outflow", "symmetry", "symmetry"),
                             u_in=(u_lattice * DX / DT, 0.0), theta_ref=-0.55)
    p.update(over)
    seeds = np.array([[0.375 * n, 0.5 * n, 10.0, 0.0]])
    return Case(f"forced_flow_{n}", p, seeds, 0.0, -0.55, steps)


def dart_seeds(nx: int, ny: int, count: int, min_spacing: float, margin: float, rmin: float, rmax: float,
               omax: float, rng: np.random.Generator, max_tries: int = 200000) -> np.ndarray:
    """Seed centres by dart throwing (uniform positions, rejected when closer
    than min_spacing to an accepted one or within margin of the edge), radii
    uniform in [rmin, rmax], orientations uniform in [0, omax)."""
    pts = []
    tries = 0
    while len(pts) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("dart throwing did not place every seed")
        x = rng.uniform(margin, nx - margin)
        y = rng.uniform(margin, ny - margin)
        if all((x - a) ** 2 + (y - b) ** 2 >= min_spacing**2 for a, b in pts):
            pts.append((x, y))
    pts = np.array(pts)
    R = rng.uniform(rmin, rmax, count)
    o = rng.uniform(0.0, omax, count)
    return np.column_stack([pts, R, o])


def multi_seed(n: int = 4096, count: int = 64, steps: int = 10000, rng_seed: int = 3,
               min_spacing: float = 200.0, **over) -> Case:
    """n x n box periodic in x with no-slip walls in y (gravity along -y),
    `count` seeds by dart throwing (spacing >= 200, margin 20), radii 6-10,
    orientations in [0, 45 deg); Delta = 0.45, eps = 0.04, buoyancy on."""
    rng = np.random.Generator(np.random.PCG64(rng_seed))
    seeds = dart_seeds(n, n, count, min_spacing, 20.0, 6.0, 10.0, math.pi / 4, rng)
    p = thermosolutal_params(n, n, eps_s=0.04, gbetaT=GBETA_T, gbetaC=GBETA_C, theta_ref=-0.45,
                             bc=("periodic", "periodic", "noslip", "noslip"))
    p.update(over)
    return Case(f"multi_seed_{n}", p, seeds, 0.0, -0.45, steps, meta={"rng_seed": rng_seed})


def batch_domains(count: int = 256, rng_seed: int = 4, lmin: int = 128, lmax: int = 1024,
                  steps: int = 5000) -> list[Case]:
    """Independent domains with side lengths log-uniform in [lmin, lmax],
    Delta in [0.3, 0.7], eps in [0.02, 0.06], orientation in [0, 45 deg),
    inflow u_x in [0, 0.02] lattice units, one seed of radius 8 at
    (0.375 L, 0.5 L), inflow left / outflow right / symmetry top and bottom."""
    rng = np.random.Generator(np.random.PCG64(rng_seed))
    L = np.rint(np.exp(rng.uniform(math.log(lmin), math.log(lmax), count))).astype(int)
    delta = rng.uniform(0.3, 0.7, count)
    eps = rng.uniform(0.02, 0.06, count)
    orient = rng.uniform(0.0, math.pi / 4, count)
    uin = rng.uniform(0.0, 0.02, count)
    cases = []
    for j in range(count):
        n = int(L[j])
        p = thermosolutal_params(n, n, eps_s=float(eps[j]), theta_ref=-float(delta[j]),
                                 bc=("inflow", "outflow", "symmetry", "symmetry"),
                                 u_in=(float(uin[j]) * DX / DT, 0.0))
        seeds = np.array([[0.375 * n, 0.5 * n, 8.0, float(orient[j])]])
        cases.append(Case(f"batch_{j}_{n}", p, seeds, 0.0, -float(delta[j]), steps))
    return cases


# -------------------------------------------------------------- random fields
def smooth_field(nx: int, ny: int, rng: np.random.Generator, modes: int = 4, amp: float = 1.0) -> np.ndarray:
    """A smooth periodic random field: a sum of `modes` x `modes` Fourier modes
    with random amplitudes decaying with wavenumber."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    out = np.zeros((ny, nx))
    for kx in range(modes):
        for ky in range(modes):
            if kx == 0 and ky == 0:
                continue
            a = rng.normal() / (kx * kx + ky * ky)
            ph = rng.uniform(0, 2 * math.pi)
            out += a * np.cos(2 * math.pi * (kx * x / nx + ky * y / ny) + ph)
    m = np.abs(out).max()
    return amp * out / (m if m > 0 else 1.0)


def random_fields(nx: int, ny: int, rng_seed: int, u_amp: float = 0.2, p_amp: float = 0.01,
                  theta0: float = -0.5, U0: float = -0.2) -> tuple[np.ndarray, np.ndarray]:
    """Random initial macroscopic fields [6, ny, nx] = (phi, U, theta, ux, uy,
    p), velocity and pressure in paper units, and a random grain-orientation
    map (four stripes of constant orientation).  phi is a smooth random level
    set passed through a steep tanh, so it spans liquid, solid and interfaces
    of a few nodes; the other fields are smooth perturbations."""
    rng = np.random.Generator(np.random.PCG64(rng_seed))
    # steep enough that every interior extremum of phi sits in a settled bulk
    # phase (|phi| > 0.9999): there grad(phi) -> 0 while d(phi)/dt ~ 0
    phi = np.tanh(8.0 * smooth_field(nx, ny, rng, 3, 1.0) + 0.3)
    U = U0 + smooth_field(nx, ny, rng, 3, 0.2)
    th = theta0 + smooth_field(nx, ny, rng, 3, 0.2)
    ux = smooth_field(nx, ny, rng, 3, u_amp)
    uy = smooth_field(nx, ny, rng, 3, u_amp)
    p = smooth_field(nx, ny, rng, 3, p_amp)
    orient = np.zeros((ny, nx))
    angles = rng.uniform(0.0, math.pi / 4, 4)
    for j in range(4):
        orient[:, j * nx // 4:(j + 1) * nx // 4] = angles[j]
    return np.stack([phi, U, th, ux, uy, p]), orient


def noise(shape, rng_seed: int, amp: float) -> np.ndarray:
    """Uniform noise in [-amp, amp] of the given shape."""
    rng = np.random.Generator(np.random.PCG64(rng_seed))
    return rng.uniform(-amp, amp, shape)


# -------------------------------------------------------------- network weights
def bf16_exact(a: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as FP64, so
    that FP64 and BF16 consumers of the same weights see the same numbers."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def unet_params(shapes, rng_seed: int, out_scale: float = 0.01) -> dict:
    """He-normal weights (standard deviation sqrt(2 / fan_in)), small random
    biases, a small output projection; every value BF16-exact.  `shapes` is
    the ordered (name, shape) list of the network definition."""
    rng = np.random.Generator(np.random.PCG64(rng_seed))
    out = {}
    for name, shape in shapes:
        if name.endswith(".W"):
            fan_in = shape[1]
            std = math.sqrt(2.0 / fan_in) * (out_scale if name.startswith("out") else 1.0)
            out[name] = bf16_exact(rng.normal(0.0, std, shape))
        else:
            out[name] = bf16_exact(rng.normal(0.0, 0.01, shape))
    return out


def surrogate_domains(count: int = 32, n: int = 256, rng_seed: int = 5, steps: int = 4000,
                      forced_flow_share: float = 0.5) -> list[Case]:
    """Training trajectories for the surrogate: n x n domains in the forced-flow
    geometry (inflow left, outflow right, symmetry top and bottom), one seed of
    radius 6-12 near (0.375 n, 0.5 n).  The first forced_flow_share of them
    take the forced-flow case's parameters (Delta = 0.55, eps = 0.05, inflow
    u_x = 0.01 lattice units, orientation 0); the rest draw them as the
    batched-domain workload does: Delta in [0.45, 0.65], eps in [0.03, 0.06],
    inflow u_x in [0, 0.02], orientation in [0, 45 deg)."""
    rng = np.random.Generator(np.random.PCG64(rng_seed))
    cases = []
    n_ff = int(round(forced_flow_share * count))
    for j in range(count):
        delta = float(rng.uniform(0.45, 0.65))
        eps = float(rng.uniform(0.03, 0.06))
        uin = float(rng.uniform(0.0, 0.02))
        orient = float(rng.uniform(0.0, math.pi / 4))
        if j < n_ff:
            delta, eps, uin, orient = 0.55, 0.05, 0.01, 0.0
        cx = 0.375 * n + float(rng.uniform(-0.05, 0.05)) * n
        cy = 0.5 * n + float(rng.uniform(-0.05, 0.05)) * n
        R = float(rng.uniform(6.0, 12.0))
        p = thermosolutal_params(n, n, eps_s=eps, theta_ref=-delta, bc=("inflow", "outflow", "symmetry", "symmetry"),
                                 u_in=(uin * DX / DT, 0.0))
        cases.append(Case(f"surrogate_{j}_{n}", p, np.array([[cx, cy, R, orient]]), 0.0, -delta, steps))
    return cases


def surrogate_training_set(n: int = 512, per_generator: int = 8, rng_seed: int = 5) -> list[Case]:
    """Training trajectories for the surrogate from the three workload
    generators, per_generator each, on n x n domains:
      - the single dendrite in forced flow (inflow left at u_x = 0.01 lattice
        units, outflow right, symmetry top and bottom; Delta = 0.55,
        eps = 0.05, orientation 0), one seed of radius 6-12 near
        (0.375 n, 0.5 n);
      - the parameter sweep's draws in the same geometry: Delta in [0.3, 0.7],
        eps in [0.02, 0.06], orientation in [0, 45 deg), inflow u_x in
        [0, 0.02], one seed of radius 8 at (0.375 n, 0.5 n);
      - crops of the multi-seed thermosolutal box: periodic in x, no-slip
        walls in y, buoyancy on, Delta = 0.45, eps = 0.04, 1-3 seeds by dart
        throwing (spacing >= n/4, margin 20), radii 6-10, orientations in
        [0, 45 deg)."""
    rng = np.random.Generator(np.random.PCG64(rng_seed))
    flow_bc = ("inflow", "outflow", "symmetry", "symmetry")
    cases = []
    for j in range(per_generator):
        cx = 0.375 * n + float(rng.uniform(-0.05, 0.05)) * n
        cy = 0.5 * n + float(rng.uniform(-0.05, 0.05)) * n
        R = float(rng.uniform(6.0, 12.0))
        p = thermosolutal_params(n, n, eps_s=0.05, theta_ref=-0.55, bc=flow_bc, u_in=(0.01 * DX / DT, 0.0))
        cases.append(Case(f"train_forced_{j}_{n}", p, np.array([[cx, cy, R, 0.0]]), 0.0, -0.55, 0))
    for j in range(per_generator):
        delta = float(rng.uniform(0.3, 0.7))
        eps = float(rng.uniform(0.02, 0.06))
        orient = float(rng.uniform(0.0, math.pi / 4))
        uin = float(rng.uniform(0.0, 0.02))
        p = thermosolutal_params(n, n, eps_s=eps, theta_ref=-delta, bc=flow_bc, u_in=(uin * DX / DT, 0.0))
        cases.append(Case(f"train_sweep_{j}_{n}", p, np.array([[0.375 * n, 0.5 * n, 8.0, orient]]), 0.0, -delta, 0))
    for j in range(per_generator):
        count = int(rng.integers(1, 4))
        seeds = dart_seeds(n, n, count, n / 4, 20.0, 6.0, 10.0, math.pi / 4, rng)
        p = thermosolutal_params(n, n, eps_s=0.04, gbetaT=GBETA_T, gbetaC=GBETA_C, theta_ref=-0.45,
                                 bc=("periodic", "periodic", "noslip", "noslip"))
        cases.append(Case(f"train_multi_{j}_{n}", p, seeds, 0.0, -0.45, 0))
    return cases


def cylinder_flow(Re: float = 40.0, nx: int = 1400, ny: int = 800, R: float = 20.0, u0: float = 0.1) -> Case:
    """Flow past a stationary cylinder (Sec. 4.1): a (70 x 40) R_s domain of
    nx x ny nodes, the disc of radius R nodes at (20 R, 20 R) as a diffuse
    circle with W0 = 0.5 dx, inflow u0 = 0.1 (lattice) on the left, outflow on
    the right, symmetry walls at the top and bottom (reading), Re = 2 u0 R / nu.
    Paper units: W0 = tau0 = 1, dx = 2 W0, dt = tau0, so nu (lattice) = 4 / Re
    for R = 20, u0 = 0.1, and s2 = 1.25 at Re = 40 as in the paper.  No
    buoyancy; the scalar fields are frozen by the flow-only stepping."""
    dx, dt = 2.0, 1.0
    nu_lu = 2.0 * u0 * R / Re
    p = thermosolutal_params(nx, ny, dx=dx, dt=dt, nu=nu_lu * dx * dx / dt, gbetaT=0.0, gbetaC=0.0,
                             bc=("inflow", "outflow", "symmetry", "symmetry"), u_in=(u0 * dx / dt, 0.0),
                             theta_ref=-0.55)
    seeds = np.array([[R * 20.0, R * 20.0, R, 0.0]])
    return Case(f"cylinder_Re{Re:g}_{nx}x{ny}", p, seeds, 0.0, -0.55, 0)
