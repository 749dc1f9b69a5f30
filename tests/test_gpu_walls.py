"""Walls with a prescribed (sliding) velocity on the GPU path, against the
oracle running the same walls and against the closed-form channel flow:

- FP64 within 1e-10 after one step and 1e-8 after 30 (2D sliding-lid
  channel, 3D dam break on a floor sliding along x and y);
- mixed accelerations within 1e-5 of max(|a_ref|, g), densities within 1e-6
  after one step;
- explicit zero wall velocities give exactly the result of walls at rest;
- a batch mixing sliding and resting tanks equals one-tank contexts exactly;
- the GPU's steady sliding-lid flow matches u = U eta (3 eta - 2) at
  mid-channel (the oracle's pin), at dp = H/20 and H/40.
"""
import numpy as np
import pytest

from paper_2603_11868_gb300 import cases

pytestmark = pytest.mark.gpu
FIELDS = ("pos", "vel", "rho", "p", "drho", "acc", "aprior")


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2603_11868_gb300 import build
    build.build()
    from paper_2603_11868_gb300 import sph as S
    S.load()
    return S


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.lib()
    return oracle


def rel(got, want):
    den = np.abs(want).max()
    return np.abs(got - want).max() / (den if den > 0 else 1.0)


def sliding_floor_3d():
    c = cases.dam_break_3d(dp=0.02, seed=5)
    wv = np.zeros_like(c.wall)
    floor = c.wall[:, 2] < 0
    wv[floor] = (0.4, -0.25, 0.0)
    c.wall_vel = wv
    return c


CASES = {"lid_2d": lambda: cases.sliding_lid_channel_2d(), "floor_3d": sliding_floor_3d}


def _run(sph, O, case, precision, steps):
    s = sph.Solver(case, precision=precision)
    s.set_option(sph.SPH_OPT_RECORD_DIAGNOSTICS, 1)
    s.step(steps)
    got = s.fields(*FIELDS)
    s.close()
    o = O.Oracle.from_case(case)
    o.step(steps)
    want = {"pos": o.field(O.POS), "vel": o.field(O.VEL), "rho": o.field(O.RHO),
            "p": o.field(O.P), "drho": o.field(O.DRHO), "acc": o.field(O.ACC),
            "aprior": o.field(O.APRIOR)}
    return got, want


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_one_step(sph, O, name):
    got, want = _run(sph, O, CASES[name](), "fp64", 1)
    for k in FIELDS:
        assert rel(got[k], want[k]) <= 1e-10, (k, rel(got[k], want[k]))


def test_fp64_thirty_steps(sph, O):
    got, want = _run(sph, O, CASES["lid_2d"](), "fp64", 30)
    for k in ("pos", "vel", "rho", "p", "drho"):
        assert rel(got[k], want[k]) <= 1e-8, (k, rel(got[k], want[k]))


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_one_step(sph, O, name):
    case = CASES[name]()
    got, want = _run(sph, O, case, "mixed", 1)
    g = max(abs(x) for x in case.gravity) or 1.0
    for k in ("acc", "aprior"):
        err = np.abs(got[k] - want[k]).max() / max(np.abs(want[k]).max(), g)
        assert err <= 1e-5, (k, err)
    assert rel(got["rho"], want["rho"]) <= 1e-6
    # the sliding walls drive the flow: the lid / floor velocity shows up
    assert np.abs(want["aprior"] - np.array(case.gravity)).max() > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_zero_wall_velocity_is_a_wall_at_rest(sph, precision):
    c = cases.dam_break_2d()
    out = []
    for wv in (None, np.zeros_like(c.wall)):
        c.wall_vel = wv
        s = sph.Solver(c, precision=precision)
        s.step(20)
        out.append(s.fields("pos", "vel", "rho"))
        s.close()
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


def test_batch_with_sliding_walls_equals_single_tanks(sph):
    cs = [cases.batched_tank(n, dp=0.02, seed=60 + k) for k, n in enumerate((500, 1200, 300))]
    for c, u in zip(cs, (0.3, 0.0, -0.2)):
        if u:
            wv = np.zeros_like(c.wall)
            wv[c.wall[:, 1] < 0, 0] = u  # sliding floor
            c.wall_vel = wv
    b = sph.Batch(cs, precision="mixed")
    b.step(25)
    f = b.fields("pos", "vel", "rho", "drho")
    for t, c in enumerate(cs):
        s = sph.Solver(c, precision="mixed")
        s.step(25)
        want = s.fields("pos", "vel", "rho", "drho")
        s.close()
        for k in want:
            assert np.array_equal(f[k][b.offsets[t]:b.offsets[t + 1]], want[k]), (t, k)
    b.close()


@pytest.mark.parametrize("dp,bar", [(0.05, 0.03), (0.025, 0.03)])
def test_sliding_lid_channel_matches_the_closed_form(sph, dp, bar):
    from test_oracle_walls import lid_profile  # same folder (pytest prepends it)
    c = cases.sliding_lid_channel_2d(dp=dp)
    s = sph.Solver(c, precision="mixed")

    def fields_at(n):
        s.step(n)
        f = s.fields("pos", "vel")
        return s.scalars()["t"], f["pos"], f["vel"]

    u, ref = lid_profile(fields_at, c, 7.5, 200)
    s.close()
    err = np.abs(u - ref).max()
    assert err <= bar * c.meta["U"], (err, u, ref)
    assert abs(u.mean()) <= 0.01 * c.meta["U"]


# --------------------------------------------------------------------------
# translating walls (sph_set_wall_translation)
def pushing_wall_3d():
    """3D dam break whose back wall (x < 0) translates into the column."""
    c = cases.dam_break_3d(dp=0.02, seed=6)
    back = c.wall[:, 0] < 0
    wv = np.zeros_like(c.wall)
    wv[back, 0] = 0.5
    c.wall_vel = wv
    c.wall_moves = back.astype(np.uint8)
    return c


TRANSLATING = {"piston_2d": lambda: cases.piston_channel_2d(V=2.0), "push_3d": pushing_wall_3d}


@pytest.mark.parametrize("name", sorted(TRANSLATING))
def test_translating_fp64_one_step(sph, O, name):
    case = TRANSLATING[name]()
    got, want = _run(sph, O, case, "fp64", 1)
    for k in FIELDS:
        if k == "p":
            # the piston's fluid starts at rest at the lattice density: after
            # one step p is round-off on both sides, so it is measured against
            # the pressure of a unit-speed impact, rho0 c0 (1 m/s)
            err = np.abs(got[k] - want[k]).max() / max(np.abs(want[k]).max(),
                                                       case.rho0 * case.c0)
        else:
            err = rel(got[k], want[k])
        assert err <= 1e-10, (k, err)


def test_translating_fp64_across_cells(sph, O):
    """130 steps: the piston crosses more than two cells, so its walls are
    binned again several times; the states and the neighbour sets agree."""
    case = TRANSLATING["piston_2d"]()
    s = sph.Solver(case, precision="fp64")
    s.step(130)
    got = s.fields("pos", "vel", "rho", "p")
    stats = s.neighbour_stats()
    t = s.scalars()["t"]
    s.close()
    o = O.Oracle.from_case(case)
    o.step(130)
    assert case.meta["V"] * t > 2.5 * 2 * case.h
    want = {"pos": o.field(O.POS), "vel": o.field(O.VEL), "rho": o.field(O.RHO),
            "p": o.field(O.P)}
    for k in want:
        assert rel(got[k], want[k]) <= 1e-8, (k, rel(got[k], want[k]))
    for g, w in zip(stats, o.neighbour_stats()):
        assert np.array_equal(g, w)


@pytest.mark.parametrize("name", sorted(TRANSLATING))
def test_translating_mixed_one_step(sph, O, name):
    case = TRANSLATING[name]()
    got, want = _run(sph, O, case, "mixed", 1)
    g = max(abs(x) for x in case.gravity) or 1.0
    for k in ("acc", "aprior"):
        err = np.abs(got[k] - want[k]).max() / max(np.abs(want[k]).max(), g)
        assert err <= 1e-5, (k, err)
    assert rel(got["rho"], want["rho"]) <= 1e-6


def test_translating_mixed_long_run_tracks_the_oracle(sph, O):
    case = TRANSLATING["piston_2d"]()
    s = sph.Solver(case, precision="mixed")
    s.step(130)
    got = s.fields("pos", "rho")
    s.close()
    o = O.Oracle.from_case(case)
    o.step(130)
    assert np.abs(got["pos"] - o.field(O.POS)).max() <= 1e-3 * case.dp
    assert rel(got["rho"], o.field(O.RHO)) <= 1e-5


def test_piston_acoustic_state_on_the_gpu(sph):
    from test_oracle_walls import piston_plateau  # same folder (pytest prepends it)
    c = cases.piston_channel_2d()
    s = sph.Solver(c, precision="mixed")
    while s.scalars()["t"] < 0.1:
        s.step(1)
    t = s.scalars()["t"]
    f = s.fields("pos", "vel", "p")
    s.close()
    plateau, ahead = piston_plateau(f["pos"], f["vel"], f["p"], c, t)
    V = c.meta["V"]
    assert abs(f["p"][plateau].mean() / (c.rho0 * c.c0 * V) - 1) < 0.03
    assert abs(f["vel"][plateau, 0].mean() / V - 1) < 0.03
    assert np.abs(f["p"][ahead]).max() < 1e-3 * c.rho0 * c.c0 * V


def test_clearing_the_translation_puts_the_walls_back(sph, O):
    case = TRANSLATING["piston_2d"]()
    s = sph.Solver(case, precision="fp64")
    s.step(40)
    sph.sph_set_wall_translation(s.ctx, None)
    s.step(5)
    got = s.fields("pos", "rho")
    s.close()
    o = O.Oracle.from_case(case)
    o.step(40)
    o.set_wall_translation(None)
    o.step(5)
    assert rel(got["pos"], o.field(O.POS)) <= 1e-10
    assert rel(got["rho"], o.field(O.RHO)) <= 1e-10


# --------------------------------------------------------------------------
# oscillating walls (sph_set_wall_motion): the shaken tank, whose walls are
# given no velocity (the motion call supplies the velocity records)
def test_oscillating_fp64_parity(sph, O):
    case = cases.shaken_tank_2d()
    for steps, tol in ((1, 1e-10), (120, 1e-8)):
        got, want = _run(sph, O, case, "fp64", steps)
        for k in ("pos", "vel", "rho", "acc"):
            assert rel(got[k], want[k]) <= tol, (steps, k, rel(got[k], want[k]))
        # the pressure tilt is small against the background pressure: compare
        # the deviation from the mean
        dp_got, dp_want = got["p"] - want["p"].mean(), want["p"] - want["p"].mean()
        assert np.abs(dp_got - dp_want).max() <= tol * 1e3 * np.abs(dp_want).max(), steps


def test_oscillating_mixed_one_step(sph, O):
    case = cases.shaken_tank_2d()
    got, want = _run(sph, O, case, "mixed", 1)
    for k in ("acc", "aprior"):
        err = np.abs(got[k] - want[k]).max() / max(np.abs(want[k]).max(), 1.0)
        assert err <= 1e-5, (k, err)
    assert rel(got["rho"], want["rho"]) <= 1e-6


def test_shaken_tank_on_the_gpu(sph):
    from test_oracle_walls import shaken_lockin  # same folder (pytest prepends it)
    c = cases.shaken_tank_2d()
    s = sph.Solver(c, precision="mixed")

    def step_fields():
        s.step(1)
        sc = s.scalars()
        f = s.fields("pos", "vel", "p", "rho")
        return sc["t"], sc["dt_ac"], f["pos"], f["vel"], f["p"], f["rho"]

    slope_ratio, vel_ratio = shaken_lockin(step_fields, c)
    s.close()
    assert abs(slope_ratio - 1) < 0.10, slope_ratio
    assert abs(vel_ratio - 1) < 0.10, vel_ratio
