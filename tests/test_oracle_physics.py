"""Pins of the oracle's interaction stages and schedule against what the
mathematics fixes independently of the oracle: conservation by antisymmetry,
reduction to the textbook SPH forms when the Riemann dissipation vanishes,
lattice consistency for linear fields, exact ballistic motion under the
kick-drift-kick scheme, wall sign conventions, and the hydrostatic column."""
import math

import numpy as np
import pytest

from paper_2603_11868_gb300 import cases


def lattice_2d(nx, ny, dp, origin=(0.0, 0.0)):
    xs = origin[0] + (np.arange(nx) + 0.5) * dp
    ys = origin[1] + (np.arange(ny) + 0.5) * dp
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], 1)


def make(oracle_mod, dim, pos, dp, h, rho0=1.0, c0=10.0, mu=0.0, g=None, wall=None,
         vel=None, rho=None, box_pad=0.5):
    lo = pos.min(0) - box_pad
    hi = pos.max(0) + box_pad
    if wall is not None and len(wall):
        lo = np.minimum(lo, wall.min(0) - box_pad)
        hi = np.maximum(hi, wall.max(0) + box_pad)
    g = np.zeros(dim) if g is None else np.asarray(g, float)
    o = oracle_mod.Oracle(dim, lo, hi, dp, h, rho0, c0, mu, c0 / 10, g)
    if wall is not None and len(wall):
        o.set_wall(wall)
    o.set_fluid(pos, vel, rho)
    return o


def pair_grad(oracle_mod, dim, h, x):
    """All pairs within 2h by brute force: i, j, grad_i W_ij (numpy + the
    pinned scalar kernel derivative)."""
    d = x[:, None, :] - x[None, :, :]
    r = np.sqrt((d ** 2).sum(-1))
    i, j = np.nonzero((r < 2 * h) & (r > 0))
    dw = np.array([oracle_mod.dW(dim, h, rr) for rr in r[i, j]])
    grad = (dw / r[i, j])[:, None] * d[i, j]
    return i, j, grad


# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_pair_forces_conserve_momentum(oracle_mod, dim):
    c = cases.random_cloud(dim, 1200, seed=30 + dim, dp=0.08, vel_scale=1.0,
                           rho_spread=0.01, c0=10.0, mu=0.05)
    o = oracle_mod.Oracle.from_case(c)
    o.pressure_relaxation(0.0)
    a = o.field(oracle_mod.ACC)
    assert np.abs(a).sum() > 0
    assert np.abs(a.sum(0)).max() < 1e-12 * np.abs(a).sum()
    o.viscous()
    av = o.field(oracle_mod.APRIOR)
    assert np.abs(av).sum() > 0
    assert np.abs(av.sum(0)).max() < 1e-12 * np.abs(av).sum()


def test_pressure_reduces_to_textbook_symmetric_gradient(oracle_mod):
    """At rest (U_L = U_R) the limiter vanishes, P* = (p_i + p_j)/2 and the
    momentum equation becomes the symmetric SPH pressure gradient
    a_i = -sum_j m (p_i + p_j) / (rho_i rho_j) grad_i W_ij."""
    c = cases.random_cloud(2, 500, seed=41, dp=0.05, rho_spread=0.02, c0=7.0)
    o = oracle_mod.Oracle.from_case(c)
    o.pressure_relaxation(0.0)
    a = o.field(oracle_mod.ACC)
    m = c.rho0 * c.dp ** 2
    rho = c.rho
    p = c.c0 ** 2 * (rho - c.rho0)
    i, j, g = pair_grad(oracle_mod, 2, c.h, c.fluid)
    ref = np.zeros_like(a)
    np.add.at(ref, i, -(m * (p[i] + p[j]) / (rho[i] * rho[j]))[:, None] * g)
    assert np.abs(a - ref).max() < 1e-11 * np.abs(ref).max()


def test_continuity_reduces_to_textbook_form(oracle_mod):
    """With equal pressures U_L - U* = (U_L - U_R)/2 and the density rate is the
    textbook continuity equation drho_i = rho_i sum_j V_j (v_i - v_j).grad_i W_ij."""
    c = cases.random_cloud(3, 700, seed=42, dp=0.08, vel_scale=0.3, c0=9.0)
    o = oracle_mod.Oracle.from_case(c)
    o.half2(0.0)
    dr = o.field(oracle_mod.DRHO)
    V = c.dp ** 3
    v = c.vel
    i, j, g = pair_grad(oracle_mod, 3, c.h, c.fluid)
    ref = np.zeros(c.n)
    np.add.at(ref, i, c.rho0 * V * ((v[i] - v[j]) * g).sum(1))
    assert np.abs(dr - ref).max() < 1e-11 * np.abs(ref).max()


# --------------------------------------------------------------------------
# lattice consistency: linear fields on the interior of a perfect lattice
DP, HF = 0.05, 1.3


def _interior(pos, nx, ny, dp, layers=3):
    x, y = pos[:, 0], pos[:, 1]
    return ((x > layers * dp) & (x < (nx - layers) * dp) &
            (y > layers * dp) & (y < (ny - layers) * dp))


def _kappa(oracle_mod, h, dp):
    # gradient consistency of the kernel on the lattice: sum_j V (y_j - y_i) dW_ij/dy_i
    # (the continuum value is 1 by integration by parts)
    pts = lattice_2d(13, 13, dp, origin=(-6.5 * dp, -6.5 * dp))
    i, j, g = pair_grad(oracle_mod, 2, h, pts)
    centre = np.argmin((pts ** 2).sum(1))
    sel = i == centre
    return np.sum(dp * dp * (pts[j[sel], 1] - pts[centre, 1]) * g[sel, 1])


def test_lattice_density_summation(oracle_mod):
    pos = lattice_2d(20, 20, DP)
    o = make(oracle_mod, 2, pos, DP, HF * DP)
    o.density_summation()
    rho = o.field(oracle_mod.RHO)
    sig = o.field(oracle_mod.SIGMA)
    inner = _interior(pos, 20, 20, DP)
    assert np.allclose(rho, 1.0, rtol=0, atol=1e-14)       # interior exact, edge clamped
    s0 = oracle_mod.sigma0(2, DP, HF * DP)
    assert np.allclose(sig[inner], s0, rtol=1e-13)
    edge = (pos.min(1) < DP) | (pos.max(1) > 19 * DP)
    assert np.all(sig[edge] < 0.9 * s0)
    # a uniformly compressed lattice reads as denser by (dp / dp')^2 (within
    # the lattice-sum error of the kernel)
    s = 0.97
    o2 = make(oracle_mod, 2, lattice_2d(20, 20, DP * s), DP, HF * DP)
    o2.density_summation()
    rho2 = o2.field(oracle_mod.RHO)[_interior(lattice_2d(20, 20, DP * s), 20, 20, DP * s)]
    assert np.allclose(rho2, 1.0 / s ** 2, rtol=0.01)


def test_lattice_pressure_gradient(oracle_mod):
    pos = lattice_2d(20, 20, DP)
    k, c0 = 3.0, 1000.0   # stiff: rho (and V_j = m / rho_j) uniform to 1e-6
    p = k * (pos[:, 1] - 0.3)
    rho = 1.0 + p / c0 ** 2
    o = make(oracle_mod, 2, pos, DP, HF * DP, c0=c0, rho=rho)
    o.pressure_relaxation(0.0)
    a = o.field(oracle_mod.ACC)
    inner = _interior(pos, 20, 20, DP)
    kappa = _kappa(oracle_mod, HF * DP, DP)
    assert 0.95 < kappa < 1.0
    # a = -grad p / rho times the lattice consistency of the kernel
    expect = -k / rho[inner] * kappa
    assert np.allclose(a[inner, 1], expect, rtol=2e-3)
    assert np.abs(a[inner, 0]).max() < 1e-3 * k


def test_lattice_divergence(oracle_mod):
    pos = lattice_2d(20, 20, DP)
    A = np.array([[0.3, 0.1], [-0.2, 0.5]])
    vel = pos @ A.T
    o = make(oracle_mod, 2, pos, DP, HF * DP, vel=vel)
    o.half2(0.0)
    dr = o.field(oracle_mod.DRHO)
    inner = _interior(pos, 20, 20, DP)
    kappa = _kappa(oracle_mod, HF * DP, DP)
    # drho / rho = -div v, with the same lattice consistency factor
    assert np.allclose(dr[inner], -np.trace(A) * kappa, rtol=2e-3)


def test_lattice_viscous_laplacian(oracle_mod):
    """v_x = y^2 has Laplacian 2; the viscous term approximates (mu/rho) lap v,
    so a_x ~ 2 mu / rho0 in the interior (kernel consistency and the 0.01h
    regulariser leave a few per cent)."""
    pos = lattice_2d(20, 20, DP)
    vel = np.zeros_like(pos)
    vel[:, 0] = pos[:, 1] ** 2
    mu = 0.01
    o = make(oracle_mod, 2, pos, DP, HF * DP, mu=mu, vel=vel)
    o.viscous()
    a = o.field(oracle_mod.APRIOR)
    inner = _interior(pos, 20, 20, DP)
    assert np.allclose(a[inner, 0], 2 * mu, rtol=0.06)
    assert np.abs(a[inner, 1]).max() < 1e-12
    # a linear shear has zero Laplacian
    vel[:, 0] = 0.7 * pos[:, 1]
    o = make(oracle_mod, 2, pos, DP, HF * DP, mu=mu, vel=vel)
    o.viscous()
    assert np.abs(o.field(oracle_mod.APRIOR)[inner]).max() < 1e-10


def test_uniform_translation_is_force_free(oracle_mod):
    c = cases.random_cloud(3, 600, seed=77, dp=0.08, mu=0.1)
    vel = np.tile([0.3, -0.2, 0.5], (c.n, 1))
    o = oracle_mod.Oracle.from_case(c, set_particles=False)
    o.set_fluid(c.fluid, vel)
    o.half2(0.0)
    assert np.all(o.field(oracle_mod.DRHO) == 0.0)
    o.viscous()
    assert np.all(o.field(oracle_mod.APRIOR) == 0.0)
    o.pressure_relaxation(0.0)
    assert np.all(o.field(oracle_mod.ACC) == 0.0)   # p = 0 everywhere


# --------------------------------------------------------------------------
def _full_box(nx, ny, dp, layers=4):
    pos = lattice_2d(nx, ny, dp)
    wall = cases.tank_walls(2, (nx * dp, ny * dp), dp, layers, open_top=False)
    return pos, wall


def test_wall_completes_lattice(oracle_mod):
    pos, wall = _full_box(16, 12, DP)
    o = make(oracle_mod, 2, pos, DP, HF * DP, wall=wall)
    o.density_summation()
    s0 = oracle_mod.sigma0(2, DP, HF * DP)
    assert np.allclose(o.field(oracle_mod.SIGMA), s0, rtol=1e-13)


def test_wall_mirror_hydrostatic_balance(oracle_mod):
    """A closed box full of fluid at the hydrostatic state: with the pressure
    mirrored into the wall along gravity, every particle (also next to the
    walls) feels the same upward pressure acceleration kappa * g."""
    nx, ny = 16, 20
    pos, wall = _full_box(nx, ny, DP)
    g, c0 = 1.0, 20.0
    H = ny * DP
    p = g * (H - pos[:, 1])
    rho = 1.0 + p / c0 ** 2
    o = make(oracle_mod, 2, pos, DP, HF * DP, c0=c0, g=(0.0, -g), wall=wall, rho=rho)
    o.pressure_relaxation(0.0)
    a = o.field(oracle_mod.ACC)
    kappa = _kappa(oracle_mod, HF * DP, DP)
    assert np.allclose(a[:, 1] * rho, kappa * g, rtol=0.01)
    assert np.abs(a[:, 0]).max() < 0.01 * g


def test_wall_viscous_and_continuity_signs(oracle_mod):
    nx, ny = 12, 12
    pos, wall = _full_box(nx, ny, DP)
    d2 = ((pos[:, None, :] - wall[None, :, :]) ** 2).sum(-1)
    touches = (d2 < (2 * HF * DP) ** 2)
    near_wall = touches.any(1)
    # uniform slip along x: only particles that see a wall are slowed (no-slip wall)
    vel = np.tile([0.5, 0.0], (len(pos), 1))
    o = make(oracle_mod, 2, pos, DP, HF * DP, mu=0.01, wall=wall, vel=vel)
    o.viscous()
    ax = o.field(oracle_mod.APRIOR)[:, 0]
    assert np.all(ax[near_wall] < 0)
    assert np.all(ax[~near_wall] == 0.0)
    # uniform motion towards the bottom wall compresses the particles that see
    # it and expands those that see the top wall
    vel = np.tile([0.0, -0.1], (len(pos), 1))
    o = make(oracle_mod, 2, pos, DP, HF * DP, wall=wall, vel=vel)
    o.half2(0.0)
    dr = o.field(oracle_mod.DRHO)
    sees_bottom = (touches & (wall[None, :, 1] < 0)).any(1)
    sees_top = (touches & (wall[None, :, 1] > ny * DP)).any(1)
    assert np.all(dr[sees_bottom] > 0) and np.all(dr[sees_top] < 0)
    assert np.all(dr[~near_wall] == 0.0)
    # with p = 0 and no gravity only the Riemann dissipation of the mirrored
    # wall state acts: it pushes particles approaching the bottom wall back up
    # and leaves those leaving the top wall alone
    o.pressure_relaxation(0.0)
    ay = o.field(oracle_mod.ACC)[:, 1]
    assert np.all(ay[sees_bottom] > 0)
    only_top = sees_top & ~(touches & (wall[None, :, 1] < ny * DP)).any(1)
    assert only_top.sum() > 0 and np.all(ay[only_top] == 0.0)
    assert np.all(ay[~near_wall] == 0.0)


# --------------------------------------------------------------------------
def test_free_particle_is_ballistic(oracle_mod):
    """An isolated particle under gravity: kick-drift-kick integrates constant
    acceleration exactly, x = x0 + v0 t + g t^2 / 2 for any step sizes."""
    g = np.array([0.0, -9.81, 0.0])
    x0 = np.array([[0.3, 0.7, 0.2]])
    v0 = np.array([[1.5, 0.4, -0.3]])
    o = oracle_mod.Oracle(3, [-5, -5, -5], [5, 5, 5], 0.01, 0.013, 1000.0, 30.0, 1e-3, 3.0, g)
    o.set_fluid(x0, v0)
    o.step(37)
    t = o.scalars()["t"]
    x = o.field(oracle_mod.POS)[0]
    v = o.field(oracle_mod.VEL)[0]
    assert np.allclose(x, x0[0] + v0[0] * t + 0.5 * g * t * t, rtol=0, atol=1e-13)
    assert np.allclose(v, v0[0] + g * t, rtol=0, atol=1e-12)
    assert o.field(oracle_mod.RHO)[0] == 1000.0


def test_dual_time_step_schedule(oracle_mod):
    """Near rest the advection step spans ceil(0.25 c0 / (0.6 U_ref)) acoustic
    steps (no clipping): 5 steps for c0 = 10 U_ref."""
    c = cases.dam_break_2d(dp=0.05)
    o = oracle_mod.Oracle.from_case(c)
    o.step(1)
    s = o.scalars()
    assert s["n_adv"] == 1
    o.step(4)
    assert o.scalars()["n_adv"] == 1
    o.step(1)
    s = o.scalars()
    assert s["n_adv"] == 2 and s["n_ac"] == 6
    assert s["tau"] == pytest.approx(s["dt_ac"], rel=1e-12)


def test_dam_break_run_invariants(oracle_mod):
    c = cases.dam_break_2d(dp=0.05)
    o = oracle_mod.Oracle.from_case(c)
    e0 = None
    for _ in range(6):
        o.step(20)
        x = o.field(oracle_mod.POS)
        v = o.field(oracle_mod.VEL)
        m = c.rho0 * c.dp ** 2
        e = 0.5 * m * (v ** 2).sum() + m * 1.0 * x[:, 1].sum()
        e0 = e if e0 is None else e0
        assert e <= e0 * (1 + 1e-3)  # no energy from nowhere
    st = o.neighbour_state()
    assert np.array_equal(np.sort(st["ids"]), np.arange(c.n))
    assert o.scalars()["flags"] == 0
    front, ke = o.front_ke()
    assert front > c.fluid[:, 0].max() and ke > 0


@pytest.mark.slow
def test_hydrostatic_column(oracle_mod):
    """Resting column, time-averaged over the last 10% of t sqrt(g/H) = 20:
    |p - rho0 g (H - y)| <= 1% of rho0 g H below the top three layers.
    Checked at h = 1.5 dp, where the kernel's lattice gradient consistency is
    within 0.3% of one (at 1.3 dp it is 0.974 and biases the slope alone)."""
    c = cases.hydrostatic_2d(dp=0.05)
    c.h = 1.5 * c.dp
    o = oracle_mod.Oracle.from_case(c)
    H, T = c.meta["H"], 20.0
    ps, ys = [], []
    while o.scalars()["t"] < T:
        o.step(50)
        if o.scalars()["t"] > 0.9 * T:
            ps.append(o.field(oracle_mod.P))
            ys.append(o.field(oracle_mod.POS)[:, 1])
    p, y = np.mean(ps, 0), np.mean(ys, 0)
    mask = y < H - 3 * c.dp
    err = np.abs(p - c.rho0 * 1.0 * (H - y))[mask]
    assert err.max() <= 0.01 * c.rho0 * 1.0 * H
