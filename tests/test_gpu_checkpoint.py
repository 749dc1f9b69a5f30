"""Checkpoint / resume on the GPU path: a run stopped mid-way, saved,
restored into a fresh context with the same setup and continued gives the
same bits as the uninterrupted run, in FP64 and in mixed precision (the
steps are deterministic), across advection steps and with the method
options and translating walls.  A checkpoint is refused by a context with a
different setup, and a buffer that is no checkpoint is refused."""
import numpy as np
import pytest

from paper_2603_11868_gb300 import cases

pytestmark = pytest.mark.gpu
FIELDS = ("pos", "vel", "rho", "drho", "p")


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


def _solver(sph, case, precision, options):
    s = sph.Solver(case, precision=precision)
    for opt, val in options:
        s.set_option(opt, val)
    return s


def _resume_equals_continuous(sph, case, precision, first, total, options=()):
    a = _solver(sph, case, precision, options)
    a.step(total)
    want = a.fields(*FIELDS)
    want_sc = a.scalars()
    a.close()
    b = _solver(sph, case, precision, options)
    b.step(first)
    buf = b.checkpoint()
    b.close()
    c = _solver(sph, case, precision, options)
    c.restore(buf)
    c.step(total - first)
    got = c.fields(*FIELDS)
    got_sc = c.scalars()
    c.close()
    for k in FIELDS:
        assert np.array_equal(got[k], want[k]), k
    for k in ("t", "n_ac", "n_adv", "dt_ad", "dt_ac"):
        assert got_sc[k] == want_sc[k], k
    return buf


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["dam_break_2d", "dam_break_3d"])
def test_resume_is_bit_identical(sph, precision, name):
    case = cases.dam_break_2d() if name == "dam_break_2d" else cases.dam_break_3d(dp=0.02)
    # 23 steps stops inside an advection step (about 4.6 acoustic steps each)
    buf = _resume_equals_continuous(sph, case, precision, 23, 60)
    assert buf.size > case.n * 40


def test_resume_with_method_options(sph):
    case = cases.dam_break_2d()
    opts = ((sph.SPH_OPT_TRANSPORT_CORRECTION, 1), (sph.SPH_OPT_REINIT_BLENDED, 1),
            (sph.SPH_OPT_DENSITY_RIEMANN, 0))
    _resume_equals_continuous(sph, case, "mixed", 17, 45, opts)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resume_with_translating_walls(sph, precision):
    _resume_equals_continuous(sph, cases.piston_channel_2d(V=2.0), precision, 37, 90)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_resume_with_oscillating_walls(sph, precision):
    _resume_equals_continuous(sph, cases.shaken_tank_2d(), precision, 41, 100)


def test_checkpoint_of_another_setup_is_refused(sph):
    a = sph.Solver(cases.dam_break_2d(), precision="mixed")
    a.step(3)
    buf = a.checkpoint()
    a.close()
    for other in (sph.Solver(cases.dam_break_2d(), precision="fp64"),
                  sph.Solver(cases.dam_break_2d(dp=0.05), precision="mixed")):
        with pytest.raises(sph.SphError):
            other.restore(buf)
        other.close()
    c = sph.Solver(cases.dam_break_2d(), precision="mixed")
    c.set_option(sph.SPH_OPT_TRANSPORT_CORRECTION, 1)
    with pytest.raises(sph.SphError):
        c.restore(buf)
    bad = buf.copy()
    bad[0] ^= 0xFF
    c.set_option(sph.SPH_OPT_TRANSPORT_CORRECTION, 0)
    with pytest.raises(sph.SphError):
        c.restore(bad)
    with pytest.raises(sph.SphError):
        c.restore(buf[:100])
    c.restore(buf)  # the right setup takes it
    c.step(1)
    c.close()


def test_corrupt_checkpoint_is_refused_on_the_host(sph):
    """Keys outside the grid or out of storage order, and ids that are no
    permutation, are caught before anything is uploaded."""
    case = cases.dam_break_2d()
    a = sph.Solver(case, precision="fp64")
    a.step(5)
    buf = a.checkpoint()
    a.close()
    n = case.n
    ids_at = buf.size - 8 * n
    keys = buf[ids_at + 4 * n:].view(np.uint32)
    ids = buf[ids_at:ids_at + 4 * n].view(np.uint32)
    s = sph.Solver(case, precision="fp64")
    for mutate in (lambda k, i: k.__setitem__(-1, 0xFFFFFFF0),
                   lambda k, i: k.__setitem__(0, k[-1] + 1),
                   lambda k, i: i.__setitem__(1, i[0])):
        bad = buf.copy()
        k = bad[ids_at + 4 * n:].view(np.uint32)
        i = bad[ids_at:ids_at + 4 * n].view(np.uint32)
        mutate(k, i)
        with pytest.raises(sph.SphError):
            s.restore(bad)
    assert keys.size == n and ids.size == n
    s.restore(buf)
    s.step(2)
    s.close()
