"""Pins of the oracle's method variants against what the mathematics fixes:

- density relaxation without the Riemann solver (U* = (U_L + U_R)/2) is the
  textbook SPH continuity equation for fluid pairs, and for a wall particle
  the continuity equation with the mirrored velocity v_R = -v_i, whatever
  the pressures;
- the blended free-surface reinitialisation reduces exactly to the clamp
  rho0 max(sigma/sigma0, 1) when the carried density is rho0, takes the
  summed density wherever that is at least the carried one, and otherwise
  moves from the summed density towards the carried one (strictly between
  the two when the carried density is above rho0, past it when below).
"""
import numpy as np
import pytest

from paper_2603_11868_gb300 import cases


def pair_grad(oracle_mod, dim, h, x, y=None):
    """Pairs (i in x, j in y) within 2h by brute force with grad_i W_ij."""
    y = x if y is None else y
    d = x[:, None, :] - y[None, :, :]
    r = np.sqrt((d ** 2).sum(-1))
    mask = (r < 2 * h) & (r > 0)
    i, j = np.nonzero(mask)
    dw = np.array([oracle_mod.dW(dim, h, rr) for rr in r[i, j]])
    return i, j, (dw / r[i, j])[:, None] * d[i, j]


@pytest.mark.parametrize("dim", [2, 3])
def test_no_riemann_continuity_is_textbook_with_unequal_pressures(oracle_mod, dim):
    c = cases.random_cloud(dim, 600, seed=60 + dim, dp=0.08, vel_scale=0.4,
                           rho_spread=0.03, c0=6.0)
    o = oracle_mod.Oracle.from_case(c)
    o.set_variant(density_riemann=False)
    o.half2(0.0)
    dr = o.field(oracle_mod.DRHO)
    m = c.rho0 * c.dp ** dim
    rho, v = c.rho, c.vel
    i, j, g = pair_grad(oracle_mod, dim, c.h, c.fluid)
    ref = np.zeros(c.n)
    np.add.at(ref, i, rho[i] * (m / rho[j]) * ((v[i] - v[j]) * g).sum(1))
    assert np.abs(dr - ref).max() < 1e-11 * np.abs(ref).max()
    # the Riemann variant differs here (unequal pressures): the pin is not vacuous
    o2 = oracle_mod.Oracle.from_case(c)
    o2.half2(0.0)
    assert np.abs(o2.field(oracle_mod.DRHO) - ref).max() > 1e-6 * np.abs(ref).max()


def test_no_riemann_wall_term_is_mirrored_continuity(oracle_mod):
    """One fluid particle moving towards a wall lattice, no gravity, p_i = 0:
    the mirrored wall state has rho_w = rho0, V_w = dp^2, v_R = -v_i, so the
    rate is rho_i sum_w V_w (v_i - v_R).grad_i W_iw."""
    dp, h = 0.05, 0.065
    xs = (np.arange(-6, 7) + 0.5) * dp
    wall = np.stack([xs, np.full_like(xs, -0.5 * dp)], 1)
    wall = np.concatenate([wall, wall - [0.0, dp], wall - [0.0, 2 * dp]])
    pos = np.array([[0.013, 0.6 * dp]])
    vel = np.array([[0.3, -0.8]])
    c = cases.Case("wall_probe", 2, dp, h, 1.0, 10.0, 0.0, 1.0, (0.0, 0.0),
                   (-1.0, -1.0), (1.0, 1.0), pos, wall, vel=vel)
    o = oracle_mod.Oracle.from_case(c)
    o.set_variant(density_riemann=False)
    o.half2(0.0)
    dr = o.field(oracle_mod.DRHO)[0]
    _, _, g = pair_grad(oracle_mod, 2, h, pos, wall)
    ref = 1.0 * (dp * dp) * ((2.0 * vel[0]) * g).sum()
    assert abs(ref) > 0
    assert abs(dr - ref) < 1e-12 * abs(ref)


def _block(dx, ny=14, nx=20, dp=0.05):
    xs = (np.arange(nx) + 0.5) * dp * dx
    ys = (np.arange(ny) + 0.5) * dp * dx
    Y, X = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([X.ravel(), Y.ravel()], 1)


def _summed(oracle_mod, pos, rho_prev, blended, dp=0.05):
    c = cases.Case("block", 2, dp, 1.3 * dp, 1.0, 10.0, 0.0, 1.0, (0.0, 0.0),
                   (-1.0, -1.0), (2.0, 2.0), pos, np.zeros((0, 2)), rho=rho_prev)
    o = oracle_mod.Oracle.from_case(c)
    o.set_variant(reinit_blended=blended)
    o.rebuild()
    o.density_summation()
    sig0 = oracle_mod.sigma0(2, dp, 1.3 * dp)
    return o.field(oracle_mod.RHO), o.field(oracle_mod.SIGMA) / sig0


@pytest.mark.parametrize("squeeze", [1.0, 0.985])
def test_blended_reinit_is_the_clamp_when_carried_density_is_rho0(oracle_mod, squeeze):
    """Free-surface block at rest (squeeze 1) and compressed (squeeze < 1, so
    the interior sums above rho0 and the surface below)."""
    pos = _block(squeeze)
    rho0 = np.ones(len(pos))
    blended, s_ratio = _summed(oracle_mod, pos, rho0, True)
    clamp, _ = _summed(oracle_mod, pos, rho0, False)
    assert (s_ratio < 1).any() and (squeeze == 1.0 or (s_ratio > 1).any())
    assert np.array_equal(blended, clamp)


def test_blended_reinit_branches(oracle_mod):
    pos = _block(0.99)
    rng = np.random.default_rng(7)
    rho_prev = 1.0 + rng.uniform(-0.02, 0.04, len(pos))
    rho, s_ratio = _summed(oracle_mod, pos, rho_prev, True)
    rho_sum = s_ratio * 1.0
    full = rho_sum >= rho_prev
    assert full.any() and (~full).any()
    # summed density wherever it is at least the carried one
    assert np.allclose(rho[full], rho_sum[full], rtol=0, atol=1e-15)
    # otherwise strictly between the summed and the carried density when the
    # carried density is above rho0 (weight rho0 / rho_prev below one)
    part = ~full & (rho_prev > 1.0)
    assert part.any()
    assert (rho[part] > rho_sum[part]).all() and (rho[part] < rho_prev[part]).all()
    # and above the carried density's summed value otherwise (weight above one)
    low = ~full & (rho_prev < 1.0)
    if low.any():
        assert (rho[low] > rho_prev[low]).all()


def test_variants_change_a_dam_break_run(oracle_mod):
    c = cases.dam_break_2d(dp=0.05)
    out = []
    for riemann, blended in ((True, False), (False, False), (True, True)):
        o = oracle_mod.Oracle.from_case(c)
        o.set_variant(density_riemann=riemann, reinit_blended=blended)
        o.step(30)
        out.append(o.field(oracle_mod.RHO))
        assert np.isfinite(out[-1]).all()
    assert not np.array_equal(out[0], out[1]) and not np.array_equal(out[0], out[2])


# --------------------------------------------------------------------------
# transport-velocity (particle-shifting) correction
def _lattice_block(n=14, dp=0.05, dim=2):
    axes = [(np.arange(n) + 0.5) * dp for _ in range(dim)]
    grid = np.meshgrid(*axes[::-1], indexing="ij")
    return np.stack([g.ravel() for g in grid[::-1]], 1)


def _shifted(oracle_mod, pos, dim=2, dp=0.05, wall=None):
    c = cases.Case("tv", dim, dp, 1.3 * dp, 1.0, 10.0, 0.0, 1.0, tuple([0.0] * dim),
                   tuple([-1.0] * dim), tuple([2.0] * dim), pos,
                   np.zeros((0, dim)) if wall is None else wall)
    o = oracle_mod.Oracle.from_case(c)
    o.rebuild()
    o.density_summation()
    before = o.field(oracle_mod.POS)
    o.transport_correction()
    return o.field(oracle_mod.POS) - before, o.field(oracle_mod.SIGMA) / oracle_mod.sigma0(
        dim, dp, 1.3 * dp)


@pytest.mark.parametrize("dim", [2, 3])
def test_transport_correction_vanishes_on_a_perfect_lattice(oracle_mod, dim):
    pos = _lattice_block(n=14 if dim == 2 else 9, dim=dim)
    d, s = _shifted(oracle_mod, pos, dim=dim)
    inner = s >= 0.95
    assert inner.any() and (~inner).any()
    # interior particles: the concentration gradient of a lattice is zero
    deep = np.all((pos > 0.05 * 3) & (pos < pos.max(0) - 0.05 * 2.5), axis=1)
    assert deep.any()
    assert np.abs(d[deep]).max() < 1e-14
    # particles without full support (the surface) never move
    assert np.abs(d[~inner]).max() == 0.0


def test_transport_correction_restores_a_displaced_particle(oracle_mod):
    """One interior particle nudged off its lattice site moves back towards it
    (away from the neighbours it crowded), by less than the nudge."""
    pos = _lattice_block(n=14)
    k = 7 * 14 + 7
    nudge = np.array([0.004, -0.0025])
    pos[k] += nudge
    d, s = _shifted(oracle_mod, pos)
    assert s[k] >= 0.95
    assert np.dot(d[k], nudge) < 0
    assert np.linalg.norm(d[k]) < np.linalg.norm(nudge)
    # the lattice neighbours it moved closer to are pushed away from it, those it
    # moved away from are drawn after it (beyond q = 0.5 the kernel slope grows
    # as particles approach)
    site = pos[k] - nudge
    r = pos - pos[k]
    near = (np.linalg.norm(pos - site, axis=1) < 1.5 * 0.05) & (np.arange(len(pos)) != k)
    closer = np.linalg.norm(r, axis=1) < np.linalg.norm(pos - site, axis=1)
    assert (near & closer).any() and (near & ~closer).any()
    for q in np.nonzero(near)[0]:
        assert (np.dot(d[q], r[q]) > 0) == closer[q], q


def test_transport_correction_runs_in_the_schedule(oracle_mod):
    c = cases.dam_break_2d(dp=0.05)
    a = oracle_mod.Oracle.from_case(c)
    a.step(12)
    b = oracle_mod.Oracle.from_case(c)
    b.set_transport_correction(True)
    b.step(12)
    pa, pb = a.field(oracle_mod.POS), b.field(oracle_mod.POS)
    assert np.isfinite(pb).all()
    assert 0 < np.abs(pa - pb).max() < 0.05 * c.dp
