"""The autotuner and mid-run option changes leave every result unchanged.

Launch configurations (block size / batch tile, radix width, neighbour lists)
only change timing: the mixed path is bit-identical across them.  The
autotuner runs its trials from a device snapshot and restores it, so a run
interrupted by sph_autotune ends exactly where an uninterrupted run ends.
"""
import numpy as np
import pytest

from paper_2603_11868_gb300 import cases

pytestmark = pytest.mark.gpu

FIELDS = ("pos", "vel", "rho", "p", "drho", "aprior")


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


def _solver_run(sph, case, plan):
    """plan: list of ("step", n) / ("opt", option, value) / ("tune", steps)."""
    s = sph.Solver(case, precision="mixed")
    tuned = None
    for item in plan:
        if item[0] == "step":
            s.step(item[1])
        elif item[0] == "opt":
            s.set_option(item[1], item[2])
        else:
            tuned = s.autotune(item[1])
    f = s.fields(*FIELDS)
    sc = s.scalars()
    s.close()
    return f, sc, tuned


def _same(a, b):
    for k in FIELDS:
        assert np.array_equal(a[k], b[k]), (k, np.abs(a[k] - b[k]).max())


def test_radix_change_mid_advection_step(sph):
    case = cases.dam_break_2d()
    ref, rsc, _ = _solver_run(sph, case, [("step", 20)])
    for bits in (11, 5):
        got, sc, _ = _solver_run(sph, case, [("step", 7), ("opt", sph.SPH_OPT_RADIX_BITS, bits),
                                             ("step", 13)])
        _same(got, ref)
        assert sc["t"] == rsc["t"]


def test_lists_switched_on_mid_advection_step(sph):
    case = cases.dam_break_2d()
    ref, _, _ = _solver_run(sph, case, [("step", 20)])
    got, _, _ = _solver_run(sph, case, [("opt", sph.SPH_OPT_NEIGHBOUR_LIST, 0), ("step", 7),
                                        ("opt", sph.SPH_OPT_NEIGHBOUR_LIST, 1), ("step", 13)])
    _same(got, ref)


@pytest.mark.parametrize("name", ["dam_break_2d", "dam_break_3d_small"])
def test_autotune_restores_the_context(sph, name):
    case = cases.dam_break_2d() if name == "dam_break_2d" else cases.dam_break_3d(dp=0.02)
    ref, rsc, _ = _solver_run(sph, case, [("step", 20)])
    got, sc, tuned = _solver_run(sph, case, [("step", 7), ("tune", 5), ("step", 13)])
    _same(got, ref)
    assert sc["t"] == rsc["t"] and sc["n_adv"] == rsc["n_adv"]
    assert tuned["block"] in (64, 96, 128, 192, 256)
    assert 5 <= tuned["radix_bits"] <= 11
    assert tuned["neighbour_list"] in (0, 1)
    assert tuned["trials"] == 1 + 4 + 6 + 1
    assert tuned["ms_per_step"] > 0


def test_batch_autotune_restores_the_batch(sph):
    cs = [cases.batched_tank(n, dp=0.02, seed=20 + k) for k, n in enumerate((300, 1500, 800))]

    def run(plan):
        b = sph.Batch(cs, precision="mixed")
        tuned = None
        for item in plan:
            if item[0] == "step":
                b.step(item[1])
            else:
                tuned = b.autotune(item[1])
        f = b.fields(*FIELDS)
        sc = b.scalars()
        b.close()
        return f, sc, tuned

    ref, rsc, _ = run([("step", 20)])
    got, sc, tuned = run([("step", 9), ("tune", 4), ("step", 11)])
    _same(got, ref)
    assert np.array_equal(sc["t"], rsc["t"]) and np.array_equal(sc["n_adv"], rsc["n_adv"])
    assert tuned["trials"] == 12 and tuned["block"] in (64, 96, 128, 192, 256)


def test_autotune_needs_particles(sph):
    ctx = sph.sph_create(2, (0, 0), (1, 1), 0.01, 0.013, 1.0, 10.0, 0.0, 1.0, (0, -1))
    with pytest.raises(sph.SphError) as e:
        sph.sph_autotune(ctx, 3)
    assert e.value.code == sph.SPH_E_STATE
    sph.sph_destroy(ctx)
