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
