"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module only places particles and states case constants; it holds none of
the method's arithmetic.  Every workload is a synthetic stand-in for the dam
breaks the paper benchmarks (section "Performance Evaluation"): fluid on a
lattice of spacing dp with seeded uniform jitter, static wall particles in
layers outside each tank face (a tank length that is not a whole number of dp
is rounded to one, so the wall lattice has no gap), and the material /
gravity constants of the case.

Workloads:
  dam_break_2d      2D dam break, tank 5.366 x 5.366, column 2.0 x 1.0 at the
                    bottom-left, dp = 0.025 (80 x 40 fluid), 4 closed wall layers,
                    rho0 = 1, g = 1, c0 = 20.
  dam_break_3d      3D dam break, tank 1.6 x 0.67 x 0.6, column 0.4 x 0.67 x 0.3,
                    3 open-top wall layers, rho0 = 1000, g = 9.81,
                    c0 = 10 sqrt(2 g H); dp = 0.01 gives 40 x 67 x 30 = 80 400
                    fluid, dp = 0.0025 gives 160 x 268 x 120 = 5 145 600.
  hydrostatic_2d    resting 2D water column in a closed tank.
  uniform_cube      N particles uniform in the unit cube, h chosen for a mean
                    of `neighbours` particles within 2h.
  batched_tanks     many independent 2D dam-break tanks of log-uniform size.
  sliding_lid_channel_2d
                    closed 2D channel, length 4 x height 1, completely filled,
                    its top wall sliding along x at U = 1 (no gravity,
                    Re = U H / nu = 10): far from the ends the steady flow is
                    the zero-net-flux Couette-Poiseuille profile
                    u = U eta (3 eta - 2), eta = y / H.
  piston_channel_2d closed 2D channel of fluid at rest (no gravity, inviscid)
                    whose left wall block translates into it at V = c0 / 20
                    from t = 0: a compression wave runs ahead at about c0
                    with p = rho0 c0 V and u = V behind it (linear acoustics).
  shaken_tank_2d    closed 2D tank, completely filled, whose walls all oscillate
                    along x with x = A sin(omega t) (no gravity): the fluid
                    follows the tank and the pressure tilts with the
                    tank's acceleration.
  dam_break_obstacle_3d
                    3D dam break whose surge hits a box obstacle on the floor
                    (the kind of test the paper's second workload is): tank
                    3.0 x 1.0 x 1.0, column 1.2 x 1.0 x 0.5 at the far end, a solid
                    0.2 x 0.4 x 0.2 box of wall particles at x = 0.6..0.8,
                    centred across the tank.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Case:
    name: str
    dim: int
    dp: float
    h: float
    rho0: float
    c0: float
    mu: float
    U_ref: float
    gravity: tuple
    lo: tuple
    hi: tuple
    fluid: np.ndarray                # (n, dim) float64, user order
    wall: np.ndarray                 # (nw, dim) float64
    vel: np.ndarray | None = None    # (n, dim) or None (rest)
    rho: np.ndarray | None = None    # (n,) or None (rho0)
    meta: dict = field(default_factory=dict)
    wall_vel: np.ndarray | None = None  # (nw, dim) prescribed wall velocity, or None (rest)
    wall_moves: np.ndarray | None = None  # (nw,) 1: the wall translates with its velocity
    wall_omega: float = 0.0              # angular frequency of translating walls' oscillation
    wall_amplitude: np.ndarray | None = None  # (nw, dim) oscillation amplitude, or None

    @property
    def n(self) -> int:
        return int(self.fluid.shape[0])

    @property
    def nw(self) -> int:
        return int(self.wall.shape[0])


def _axis_coords(n_in: int, length: float, dp: float, lo_idx: int, hi_idx: int) -> np.ndarray:
    """Lattice coordinates along one axis for indices lo_idx..hi_idx-1.
    Indices 0..n_in-1 sit inside the tank at (i + 1/2) dp; indices below 0 sit
    outside the low face at (i + 1/2) dp; indices n_in and above sit outside
    the high face at length + (i - n_in + 1/2) dp (length = n_in dp, see
    lattice_length)."""
    i = np.arange(lo_idx, hi_idx, dtype=np.float64)
    inside = (i + 0.5) * dp
    above = length + (i - n_in + 0.5) * dp
    return np.where(i < n_in, inside, above)


def lattice_length(length: float, dp: float) -> float:
    """A tank length on the particle lattice: unchanged when it is a whole
    number of dp, else rounded to the nearest whole number of dp (at least
    one).  A high face placed off the lattice would leave the walls normal to
    it with a gap of dp to 2 dp next to that face, wide enough for fluid to
    leak through the floor at the far corner once the surge arrives."""
    n = max(1, int(round(length / dp)))
    return length if abs(length / dp - n) <= 1e-9 else n * dp


def tank_walls(dim: int, tank, dp: float, layers: int, open_top: bool) -> np.ndarray:
    """Wall particles: every lattice point of the tank grown by `layers` on each
    face (not above the top face when open_top) that lies outside the tank.
    Each tank length is taken on the lattice first (lattice_length), so the
    wall lattice has spacing dp everywhere."""
    tank = [lattice_length(L, dp) for L in tank]
    n_in = [int(math.floor(L / dp + 1e-9)) for L in tank]
    ranges = []
    for k in range(dim):
        top = n_in[k] if (open_top and k == dim - 1) else n_in[k] + layers
        ranges.append((-layers, top))
    idx = np.meshgrid(*[np.arange(a, b) for a, b in ranges], indexing="ij")
    idx = [a.ravel() for a in idx]
    inside = np.ones_like(idx[0], dtype=bool)
    for k in range(dim):
        inside &= (idx[k] >= 0) & (idx[k] < n_in[k])
    keep = ~inside
    cols = []
    for k in range(dim):
        coords = _axis_coords(n_in[k], tank[k], dp, ranges[k][0], ranges[k][1])
        cols.append(coords[idx[k][keep] - ranges[k][0]])
    return np.stack(cols, axis=1)


def fluid_block(dim: int, origin, size, dp: float, jitter: float, rng) -> np.ndarray:
    """Lattice block of fluid at (i + 1/2) dp from `origin`, x fastest, plus a
    uniform jitter in [-jitter dp, +jitter dp] per component."""
    counts = [int(round(s / dp)) for s in size]
    axes = [origin[k] + (np.arange(counts[k]) + 0.5) * dp for k in range(dim)]
    grid = np.meshgrid(*axes[::-1], indexing="ij")  # slowest axis first
    pts = np.stack([g.ravel() for g in grid[::-1]], axis=1)
    if jitter:
        pts = pts + rng.uniform(-jitter * dp, jitter * dp, size=pts.shape)
    return np.ascontiguousarray(pts)


def _domain(dim, tank, dp, layers, headroom):
    lo = tuple(-(layers + 1) * dp for _ in range(dim))
    hi = [tank[k] + (layers + 1) * dp for k in range(dim)]
    hi[dim - 1] += headroom
    return lo, tuple(hi)


def dam_break_2d(dp: float = 0.025, seed: int = 0, jitter: float = 0.01, layers: int = 4,
                 tank=(5.366, 5.366), column=(2.0, 1.0), rho0: float = 1.0, g: float = 1.0,
                 c0: float = 20.0) -> Case:
    """Closed 2D tank, water column at the bottom-left corner."""
    rng = np.random.default_rng(seed)
    fluid = fluid_block(2, (0.0, 0.0), column, dp, jitter, rng)
    wall = tank_walls(2, tank, dp, layers, open_top=False)
    lo, hi = _domain(2, tank, dp, layers, 0.0)
    U_ref = c0 / 10.0
    H = column[1]
    mu = rho0 * U_ref * H / 1000.0      # Reynolds number 1000 on (U_ref, H)
    return Case("dam_break_2d", 2, dp, 1.3 * dp, rho0, c0, mu, U_ref, (0.0, -g), lo, hi,
                fluid, wall, meta=dict(tank=tank, column=column, layers=layers, seed=seed))


def dam_break_3d(dp: float = 0.01, seed: int = 1, jitter: float = 0.01, layers: int = 3,
                 tank=(1.6, 0.67, 0.6), column=(0.4, 0.67, 0.3), rho0: float = 1000.0,
                 g: float = 9.81, mu: float = 1.0e-3) -> Case:
    """Open-top 3D tank; z is the vertical axis.  c0 = 10 sqrt(2 g H)."""
    rng = np.random.default_rng(seed)
    fluid = fluid_block(3, (0.0, 0.0, 0.0), column, dp, jitter, rng)
    wall = tank_walls(3, tank, dp, layers, open_top=True)
    lo, hi = _domain(3, tank, dp, layers, 0.25 * tank[2])
    H = column[2]
    c0 = 10.0 * math.sqrt(2.0 * g * H)
    return Case("dam_break_3d", 3, dp, 1.3 * dp, rho0, c0, mu, c0 / 10.0, (0.0, 0.0, -g), lo,
                hi, fluid, wall, meta=dict(tank=tank, column=column, layers=layers, seed=seed))


def hydrostatic_2d(dp: float = 0.05, width: float = 1.0, height: float = 1.0,
                   tank_height: float = 1.2, layers: int = 4, seed: int = 5,
                   rho0: float = 1.0, g: float = 1.0, c0: float = 20.0,
                   mu: float | None = None) -> Case:
    """Resting column filling the tank width in a closed tank; the initial
    density carries the hydrostatic profile rho0 + rho0 g (H - y) / c0^2."""
    rng = np.random.default_rng(seed)
    tank = (width, tank_height)
    fluid = fluid_block(2, (0.0, 0.0), (width, height), dp, 0.0, rng)
    wall = tank_walls(2, tank, dp, layers, open_top=False)
    lo, hi = _domain(2, tank, dp, layers, 0.0)
    U_ref = c0 / 10.0
    if mu is None:
        mu = rho0 * U_ref * height / 100.0
    Hn = round(height / dp) * dp
    rho = rho0 + rho0 * g * (Hn - fluid[:, 1]) / (c0 * c0)
    return Case("hydrostatic_2d", 2, dp, 1.3 * dp, rho0, c0, mu, U_ref, (0.0, -g), lo, hi,
                fluid, wall, rho=np.ascontiguousarray(rho),
                meta=dict(tank=tank, H=Hn, layers=layers))


def uniform_cube(n: int = 1 << 24, seed: int = 3, neighbours: float = 57.0) -> Case:
    """Uniform random particles in [0,1)^3; h such that the expected number of
    other particles within 2h is `neighbours` (n (4/3) pi (2h)^3 = neighbours)."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, 3))
    two_h = (neighbours / (n * 4.0 / 3.0 * math.pi)) ** (1.0 / 3.0)
    h = 0.5 * two_h
    dp = n ** (-1.0 / 3.0)
    return Case("uniform_cube", 3, dp, h, 1.0, 10.0, 0.0, 1.0, (0.0, 0.0, 0.0),
                (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), np.ascontiguousarray(pts),
                np.zeros((0, 3)), meta=dict(seed=seed, neighbours=neighbours))


def random_cloud(dim: int, n: int, seed: int, box: float = 1.0, dp: float = 0.05,
                 h_factor: float = 1.3, vel_scale: float = 0.0, rho_spread: float = 0.0,
                 rho0: float = 1.0, c0: float = 10.0, mu: float = 0.0,
                 gravity=None) -> Case:
    """Small disordered cloud (no walls) for invariant tests: positions uniform
    in a box, optional random velocities and densities."""
    rng = np.random.default_rng(seed)
    pts = rng.random((n, dim)) * box
    vel = rng.normal(size=(n, dim)) * vel_scale if vel_scale else None
    rho = rho0 * (1.0 + rho_spread * rng.uniform(-1, 1, n)) if rho_spread else None
    g = tuple(gravity) if gravity is not None else tuple(0.0 for _ in range(dim))
    margin = 0.1 * box
    return Case("random_cloud", dim, dp, h_factor * dp, rho0, c0, mu, c0 / 10.0, g,
                tuple(-margin for _ in range(dim)), tuple(box + margin for _ in range(dim)),
                np.ascontiguousarray(pts), np.zeros((0, dim)), vel=vel, rho=rho)


def batched_tank_sizes(n_tanks: int = 256, seed: int = 4, n_min: int = 1000,
                       n_max: int = 64000):
    """Per-tank fluid counts, log-uniform in [n_min, n_max]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(n_min), math.log(n_max), n_tanks))


def batched_tank(n_target: float, dp: float = 0.01, seed: int = 0, layers: int = 4,
                 jitter: float = 0.01) -> Case:
    """One tank of the batch: a 2:1 column of about n_target particles
    (H = dp sqrt(n/2), W = 2H) in a closed square tank of side 2.683 W;
    rho0 = 1, g = 1, c0 = 20 sqrt(H) (so c0 = 10 U_ref with U_ref = 2 sqrt(g H)),
    Reynolds number 1000."""
    ny = max(4, int(round(math.sqrt(n_target / 2.0))))
    nx = 2 * ny
    H, Wc = ny * dp, nx * dp
    side = 2.683 * Wc
    c0 = 20.0 * math.sqrt(H)
    case = dam_break_2d(dp=dp, seed=seed, jitter=jitter, layers=layers, tank=(side, side),
                        column=(Wc, H), rho0=1.0, g=1.0, c0=c0)
    case.name = "batched_tank"
    return case


def box_particles(dim: int, lo, size, dp: float) -> np.ndarray:
    """Lattice points (i + 1/2) dp filling a solid box from corner `lo`."""
    return fluid_block(dim, lo, size, dp, 0.0, None)


def dam_break_obstacle_3d(dp: float = 0.02, seed: int = 7, jitter: float = 0.01,
                          layers: int = 3, tank=(3.0, 1.0, 1.0), column=(1.2, 1.0, 0.5),
                          box=(0.2, 0.4, 0.2), box_x: float = 0.6, rho0: float = 1000.0,
                          g: float = 9.81, mu: float = 1.0e-3) -> Case:
    """Open-top 3D tank; the column fills the far end (x from tank_x -
    column_x), the surge runs towards x = 0 and meets a solid box of wall
    particles standing on the floor.  c0 = 10 sqrt(2 g H)."""
    rng = np.random.default_rng(seed)
    x0 = tank[0] - column[0]
    fluid = fluid_block(3, (x0, 0.0, 0.0), column, dp, jitter, rng)
    walls = tank_walls(3, tank, dp, layers, open_top=True)
    obstacle = box_particles(3, (box_x, 0.5 * (tank[1] - box[1]), 0.0), box, dp)
    wall = np.ascontiguousarray(np.concatenate([walls, obstacle]))
    lo, hi = _domain(3, tank, dp, layers, 0.25 * tank[2])
    H = column[2]
    c0 = 10.0 * math.sqrt(2.0 * g * H)
    return Case("dam_break_obstacle_3d", 3, dp, 1.3 * dp, rho0, c0, mu, c0 / 10.0,
                (0.0, 0.0, -g), lo, hi, fluid, wall,
                meta=dict(tank=tank, column=column, box=box, box_x=box_x, layers=layers,
                          seed=seed, n_obstacle=len(obstacle)))


def sliding_lid_channel_2d(dp: float = 0.05, length: float = 4.0, height: float = 1.0,
                           U: float = 1.0, nu: float = 0.1, c0: float = 20.0,
                           compression: float = 1.004, layers: int = 4,
                           rho0: float = 1.0) -> Case:
    """Closed 2D channel filled with fluid at rest; the wall layers above the
    top face (corners included) slide along x at U, the others rest.  The
    fluid lattice is `compression` times finer than dp, centred in the
    channel, so the summed density starts above rho0 everywhere: the
    background pressure c0^2 rho0 (compression^2 - 1) keeps the pressure
    positive along the channel, where the free-surface clamp of the density
    summation would otherwise flatten the low-pressure half."""
    nx, ny = int(round(length / dp)), int(round(height / dp))
    dpf = dp / compression
    xs = 0.5 * (length - nx * dpf) + (np.arange(nx) + 0.5) * dpf
    ys = 0.5 * (height - ny * dpf) + (np.arange(ny) + 0.5) * dpf
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    fluid = np.ascontiguousarray(np.stack([X.ravel(), Y.ravel()], axis=1))
    tank = (length, height)
    wall = tank_walls(2, tank, dp, layers, open_top=False)
    wall_vel = np.zeros_like(wall)
    wall_vel[wall[:, 1] > height, 0] = U
    lo, hi = _domain(2, tank, dp, layers, 0.0)
    return Case("sliding_lid_channel_2d", 2, dp, 1.3 * dp, rho0, c0, nu * rho0, c0 / 10.0,
                (0.0, 0.0), lo, hi, fluid, wall,
                meta=dict(tank=tank, U=U, H=height, L=length, nu=nu, layers=layers),
                wall_vel=np.ascontiguousarray(wall_vel))


def piston_channel_2d(dp: float = 0.05, length: float = 4.0, height: float = 0.5,
                      V: float = 1.0, c0: float = 20.0, layers: int = 4,
                      rho0: float = 1.0, mu: float = 0.0) -> Case:
    """Closed 2D channel filled with fluid at rest on the lattice; the wall
    layers left of x = 0 (corners included) translate along +x at V from
    t = 0 (wall_moves), the others rest.  No gravity."""
    nx, ny = int(round(length / dp)), int(round(height / dp))
    fluid = fluid_block(2, (0.0, 0.0), (nx * dp, ny * dp), dp, 0.0, None)
    tank = (length, height)
    wall = tank_walls(2, tank, dp, layers, open_top=False)
    piston = wall[:, 0] < 0
    wall_vel = np.zeros_like(wall)
    wall_vel[piston, 0] = V
    lo, hi = _domain(2, tank, dp, layers, 0.0)
    return Case("piston_channel_2d", 2, dp, 1.3 * dp, rho0, c0, mu, c0 / 10.0, (0.0, 0.0),
                lo, hi, np.ascontiguousarray(fluid), wall,
                meta=dict(tank=tank, V=V, L=length, H=height, layers=layers),
                wall_vel=np.ascontiguousarray(wall_vel),
                wall_moves=piston.astype(np.uint8))


def shaken_tank_2d(dp: float = 0.025, length: float = 1.0, height: float = 0.5,
                   A: float = 0.01, omega: float = 2.0 * math.pi, c0: float = 20.0,
                   compression: float = 1.005, layers: int = 4, rho0: float = 1.0) -> Case:
    """Closed 2D tank filled with fluid (lattice `compression` times finer
    than dp, so the pressure stays positive); every wall particle translates
    with x_w(t) = x_w(0) + A sin(omega t) e_x, and the fluid starts with the
    tank's velocity A omega e_x.  No gravity, inviscid.  The domain leaves
    room for the walls' swing."""
    nx, ny = int(round(length / dp)), int(round(height / dp))
    dpf = dp / compression
    xs = 0.5 * (length - nx * dpf) + (np.arange(nx) + 0.5) * dpf
    ys = 0.5 * (height - ny * dpf) + (np.arange(ny) + 0.5) * dpf
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    fluid = np.ascontiguousarray(np.stack([X.ravel(), Y.ravel()], axis=1))
    tank = (length, height)
    wall = tank_walls(2, tank, dp, layers, open_top=False)
    lo, hi = _domain(2, tank, dp, layers, 0.0)
    lo = (lo[0] - 2 * abs(A) - dp, lo[1])
    hi = (hi[0] + 2 * abs(A) + dp, hi[1])
    vel = np.tile([A * omega, 0.0], (len(fluid), 1))
    amp = np.ascontiguousarray(np.tile([A, 0.0], (len(wall), 1)))
    return Case("shaken_tank_2d", 2, dp, 1.3 * dp, rho0, c0, 0.0, c0 / 10.0, (0.0, 0.0), lo,
                hi, fluid, wall, vel=np.ascontiguousarray(vel),
                meta=dict(tank=tank, L=length, H=height, A=A, omega=omega, layers=layers),
                wall_vel=np.zeros_like(wall), wall_moves=np.ones(len(wall), np.uint8),
                wall_omega=omega, wall_amplitude=amp)
