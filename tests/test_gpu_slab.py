"""The slab decomposition (paper_2603_11868_gb300/slab.py) on the GPU: ranks
of library contexts on one device, driven in one process (each rank's
kernels run one after the other; nothing waits across ranks inside a
kernel), against a single context of the same case:
  * FP64: every field of every particle within 1e-10 relative after many
    acoustic steps with particles crossing the cuts; the same steps and time;
  * mixed precision: within the bars below (the ranks sum in their own
    storage order, so float roundings differ from the single context's);
  * the per-step ghost exchange through device rows (the form NCCL moves)
    equals the exchange through host arrays bitwise.
"""
import numpy as np
import pytest

from paper_2603_11868_gb300 import cases

pytestmark = pytest.mark.gpu


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


def _moving(case, u):
    v = np.zeros_like(case.fluid)
    v[:, 0] = u
    case.vel = v
    return case


CASES = {
    "dam_break_2d_moving": lambda: _moving(cases.dam_break_2d(), 2.0),
    "dam_break_3d_moving": lambda: _moving(cases.dam_break_3d(dp=0.02, seed=1), 1.5),
}


def _decomposed(case, world, steps, precision, device_rows=False):
    from paper_2603_11868_gb300 import slab
    ranks = [slab.SlabRank(case, k, world,
                           slab.LibraryEngine(case, precision, device_rows=device_rows))
             for k in range(world)]
    slab.run_in_process(ranks, steps)
    out = {k: np.full((case.n, case.dim) if k in ("pos", "vel") else case.n, np.nan)
           for k in ("pos", "vel", "rho")}
    owners = np.zeros(case.n, np.int64)
    sched = [r.engine.schedule() for r in ranks]
    for r in ranks:
        gid, st = r.owned_state()
        owners[gid] += 1
        for k in out:
            out[k][gid] = st[k]
        r.engine.close()
    assert np.all(owners == 1)
    return out, sched


def _single(sph, case, steps, precision):
    s = sph.Solver(case, precision=precision)
    s.step(steps)
    f = s.fields("pos", "vel", "rho")
    sc = s.scalars()
    s.close()
    return f, sc


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name,world,steps", [("dam_break_2d_moving", 2, 60),
                                              ("dam_break_2d_moving", 3, 40),
                                              ("dam_break_3d_moving", 2, 30)])
def test_fp64_slabs_equal_one_context(sph, name, world, steps):
    case = CASES[name]()
    got, sched = _decomposed(case, world, steps, "fp64")
    want, sc = _single(sph, case, steps, "fp64")
    for k in ("pos", "vel", "rho"):
        assert _rel(got[k], want[k]) <= 1e-10, (k, _rel(got[k], want[k]))
    for s in sched:
        assert s["n_ac"] == sc["n_ac"] == steps and s["n_adv"] == sc["n_adv"]
        assert abs(s["t"] - sc["t"]) <= 1e-12 * sc["t"]
    assert sc["n_adv"] >= 3


@pytest.mark.parametrize("name,world,steps", [("dam_break_2d_moving", 2, 60),
                                              ("dam_break_3d_moving", 2, 30)])
def test_mixed_slabs_track_one_context(sph, name, world, steps):
    case = CASES[name]()
    got, sched = _decomposed(case, world, steps, "mixed")
    want, sc = _single(sph, case, steps, "mixed")
    e_pos = np.abs(got["pos"] - want["pos"]).max() / case.dp
    e_vel, e_rho = _rel(got["vel"], want["vel"]), _rel(got["rho"], want["rho"])
    print(f"\n{name}, {world} slabs, {steps} steps, mixed: pos {e_pos:.2e} dp, vel {e_vel:.2e}, "
          f"rho {e_rho:.2e}")
    assert e_pos <= 1e-5 and e_vel <= 1e-5 and e_rho <= 3e-7
    for s in sched:
        assert s["n_ac"] == sc["n_ac"] and s["n_adv"] == sc["n_adv"]


def test_device_row_exchange_equals_host_exchange(sph):
    case = CASES["dam_break_3d_moving"]()
    host, _ = _decomposed(case, 2, 25, "mixed", device_rows=False)
    dev, _ = _decomposed(case, 2, 25, "mixed", device_rows=True)
    for k in host:
        assert np.array_equal(host[k], dev[k]), k


def test_state_and_schedule_entry_points(sph):
    """The C ABI's state-by-id-range and schedule calls round-trip, refuse bad
    ranges, and set the schedule only at an advection-step boundary."""
    case = cases.dam_break_2d(dp=0.05)
    s = sph.Solver(case, precision="fp64")
    s.step(3)
    st = sph.sph_get_state_range(s.ctx, 5, 20, 2)
    f = s.fields("pos", "vel", "rho", "drho", "aprior")
    for k in ("pos", "vel", "rho", "drho", "aprior"):
        assert np.array_equal(st[k], f[k][5:25]), k
    st2 = {k: v * 1.0 for k, v in st.items()}
    st2["rho"] = st["rho"] + 1.0
    sph.sph_put_state_range(s.ctx, 5, st2)
    assert np.array_equal(s.field("rho")[5:25], st["rho"] + 1.0)
    with pytest.raises(sph.SphError) as e:
        sph.sph_get_state_range(s.ctx, case.n - 3, 10, 2)
    assert e.value.code == sph.SPH_E_INVALID
    sc = sph.sph_get_schedule(s.ctx)
    assert sc["n_ac"] == 3 and sc["started"] == 1
    bad = dict(sc, tau=0.0, dt_ad=1.0)
    with pytest.raises(sph.SphError) as e:
        sph.sph_set_schedule(s.ctx, bad)
    assert e.value.code == sph.SPH_E_INVALID
    good = dict(sc, tau=2.0, dt_ad=1.0, t=5.0)
    sph.sph_set_schedule(s.ctx, good)
    back = sph.sph_get_schedule(s.ctx)
    assert back["t"] == 5.0 and back["tau"] == 2.0
    v2 = sph.sph_owned_vmax2(s.ctx, case.n)
    vel = s.field("vel")
    assert v2 == pytest.approx(float((vel ** 2).sum(1).max()), rel=1e-15)
    sph.sph_set_vmax2(s.ctx, 0.25)
    assert sph.sph_get_schedule(s.ctx)["vmax2"] == 0.25
    s.step(1)  # the next step begins an advection step from the set schedule
    assert sph.sph_get_schedule(s.ctx)["n_adv"] == sc["n_adv"] + 1
    s.close()
