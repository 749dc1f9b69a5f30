"""Pins of the oracle's wall terms with a prescribed (sliding) wall velocity:

- Galilean invariance: giving every fluid and wall particle the same velocity
  V changes neither the pressure acceleration, nor the density rate, nor the
  viscous force (which stays g exactly), since only velocity differences and
  the mirrored wall state v_R = 2 v_w - v_i = V enter;
- the closed-form steady flow of a long closed channel under a sliding lid:
  far from the ends the flow is parallel with zero net flux, so the momentum
  balance mu u'' = dp/dx with u(0) = 0, u(H) = U and zero flux gives
  u = U eta (3 eta - 2), eta = y / H (lubrication / Couette-Poiseuille).
  This pins the viscous operator, the no-slip wall term (the mirrored wall
  velocity) and the wall velocity itself against the mathematics.
"""
import numpy as np
import pytest

from paper_2603_11868_gb300 import cases


def _jittered_box(dim, n_side, dp, seed, layers=4):
    rng = np.random.default_rng(seed)
    tank = tuple([n_side * dp] * dim)
    fluid = cases.fluid_block(dim, tuple([0.0] * dim), tank, dp, 0.05, rng)
    wall = cases.tank_walls(dim, tank, dp, layers, open_top=False)
    lo, hi = cases._domain(dim, tank, dp, layers, 0.0)
    rho = 1.0 + 0.01 * rng.uniform(-1.0, 1.0, len(fluid))
    return fluid, wall, lo, hi, rho


def _stages(oracle_mod, dim, fluid, wall, lo, hi, rho, vel, wall_vel, g):
    dp = 0.05
    c = cases.Case("box", dim, dp, 1.3 * dp, 1.0, 10.0, 0.02, 1.0, g, lo, hi, fluid, wall,
                   vel=vel, rho=rho, wall_vel=wall_vel)
    o = oracle_mod.Oracle.from_case(c)
    o.viscous()
    o.pressure_relaxation(0.0)
    o.half2(0.0)
    return (o.field(oracle_mod.APRIOR), o.field(oracle_mod.ACC), o.field(oracle_mod.DRHO))


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_motion_with_the_walls_changes_nothing(oracle_mod, dim):
    n_side = 14 if dim == 2 else 7
    fluid, wall, lo, hi, rho = _jittered_box(dim, n_side, 0.05, seed=80 + dim)
    g = (0.0, -1.0) if dim == 2 else (0.0, 0.0, -1.0)
    V = np.array([0.3, -0.2, 0.25][:dim])
    rest = _stages(oracle_mod, dim, fluid, wall, lo, hi, rho, None, None, g)
    moving = _stages(oracle_mod, dim, fluid, wall, lo, hi, rho,
                     np.tile(V, (len(fluid), 1)), np.tile(V, (len(wall), 1)), g)
    # viscous: every velocity difference is exactly zero in both runs
    assert np.array_equal(moving[0], rest[0])
    assert np.array_equal(rest[0], np.tile(np.array(g), (len(fluid), 1)))
    # pressure and density relaxation: equal up to rounding
    for k in (1, 2):
        scale = np.abs(rest[k]).max()
        assert scale > 0
        assert np.abs(moving[k] - rest[k]).max() <= 1e-11 * scale, k
    # the wall terms are exercised: a moving fluid next to walls at rest differs
    still = _stages(oracle_mod, dim, fluid, wall, lo, hi, rho,
                    np.tile(V, (len(fluid), 1)), None, g)
    assert np.abs(still[0] - rest[0]).max() > 1e-3
    assert np.abs(still[2] - rest[2]).max() > 1e-3 * np.abs(rest[2]).max()


def lid_profile(fields_at, case, t_end, step):
    """Bin-averaged u(eta) over |x - L/2| < H/2 and the last 30 % of the run;
    fields_at(n) advances n steps and returns (t, pos, vel)."""
    L, H = case.meta["L"], case.meta["H"]
    bins = np.linspace(0.0, 1.0, 11)
    acc, cnt = np.zeros(10), np.zeros(10)
    t = 0.0
    while t < t_end:
        t, pos, vel = fields_at(step)
        if t > 0.7 * t_end:
            m = np.abs(pos[:, 0] - 0.5 * L) < 0.5 * H
            b = np.clip(np.digitize(pos[m, 1] / H, bins) - 1, 0, 9)
            np.add.at(acc, b, vel[m, 0])
            np.add.at(cnt, b, 1)
    u = acc / cnt
    a, b = bins[:-1], bins[1:]
    # the closed form averaged over each bin: mean of U eta (3 eta - 2)
    ref = case.meta["U"] * ((b ** 3 - a ** 3) - (b ** 2 - a ** 2)) / (b - a)
    return u, ref


@pytest.mark.slow
def test_sliding_lid_channel_matches_the_closed_form(oracle_mod):
    c = cases.sliding_lid_channel_2d()
    o = oracle_mod.Oracle.from_case(c)

    def fields_at(n):
        o.step(n)
        return o.scalars()["t"], o.field(oracle_mod.POS), o.field(oracle_mod.VEL)

    u, ref = lid_profile(fields_at, c, 7.5, 200)
    err = np.abs(u - ref).max()
    assert err <= 0.03 * c.meta["U"], (err, u, ref)
    # zero net flux through the mid-channel section
    assert abs(u.mean()) <= 0.01 * c.meta["U"]
