"""GPU parity of batches of independent tanks (sph_create_batch / sph_batch_*).

Each tank of a batch must compute what the FP64 oracle computes for that tank
alone, on its own schedule:
  - the neighbour structure of every tank after the initial sort and after
    rebuilds: bit-exact keys, user ids and cell offsets;
  - the FP64 batch after one step: every field within 1e-10 relative; after
    40 steps (tanks at different advection-step counts) within 1e-8, with the
    tank's own step counts and times;
  - the mixed batch after one step: accelerations within 1e-5 of
    max(|a_ref|, g), as for one tank;
  - and the batch must equal one-tank contexts of the same tanks exactly
    (the same kernels walk each tank's tiles).
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


@pytest.fixture(scope="module")
def O():
    from oracle import oracle
    oracle.lib()
    return oracle


def rel(got, want):
    den = np.abs(want).max()
    return np.abs(got - want).max() / (den if den > 0 else 1.0)


def tanks(sizes=(300, 1200, 2600, 700), dp=0.02, seed0=10):
    """Small tanks of the batched workload (2:1 columns in closed square tanks,
    c0 = 20 sqrt(H)): different sizes give different wave speeds and so
    different schedules."""
    return [cases.batched_tank(n, dp=dp, seed=seed0 + k) for k, n in enumerate(sizes)]


FIELDS = ("pos", "vel", "rho", "p", "drho", "acc", "aprior", "sigma")


def _oracle_fields(o, O):
    return {"pos": o.field(O.POS), "vel": o.field(O.VEL), "rho": o.field(O.RHO),
            "p": o.field(O.P), "drho": o.field(O.DRHO), "acc": o.field(O.ACC),
            "aprior": o.field(O.APRIOR), "sigma": o.field(O.SIGMA)}


def _batch(sph, cs, precision, steps, graph=True):
    b = sph.Batch(cs, precision=precision)
    b.set_option(sph.SPH_OPT_RECORD_DIAGNOSTICS, 1)
    b.set_option(sph.SPH_OPT_USE_GRAPH, 1 if graph else 0)
    b.step(steps)
    f = b.fields(*FIELDS)
    sc = b.scalars()
    out = [{k: v[b.offsets[t]:b.offsets[t + 1]] for k, v in f.items()} for t in range(b.tanks)]
    b.close()
    return out, sc


# --------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_initial_neighbour_state_bit_exact(sph, O, precision):
    cs = tanks()
    b = sph.Batch(cs, precision=precision)
    for t, c in enumerate(cs):
        got = b.neighbour_state(t)
        want = O.Oracle.from_case(c).neighbour_state()
        for k in ("keys", "ids", "cell_begin"):
            assert np.array_equal(got[k], want[k]), (t, k)
    b.close()


def test_neighbour_state_after_rebuilds_bit_exact(sph, O):
    """After 23 steps every tank has rebuilt several times on its own schedule."""
    cs = tanks()
    b = sph.Batch(cs, precision="fp64")
    b.step(23)
    sc = b.scalars()
    for t, c in enumerate(cs):
        o = O.Oracle.from_case(c)
        o.step(23)
        assert o.scalars()["n_adv"] == sc["n_adv"][t]
        got, want = b.neighbour_state(t), o.neighbour_state()
        for k in ("keys", "ids", "cell_begin"):
            assert np.array_equal(got[k], want[k]), (t, k)
    b.close()


def test_fp64_one_step(sph, O):
    cs = tanks()
    got, sc = _batch(sph, cs, "fp64", 1)
    for t, c in enumerate(cs):
        o = O.Oracle.from_case(c)
        o.step(1)
        want = _oracle_fields(o, O)
        for k in FIELDS:
            assert rel(got[t][k], want[k]) <= 1e-10, (t, k, rel(got[t][k], want[k]))
        osc = o.scalars()
        assert sc["dt_ac"][t] == osc["dt_ac"] and sc["dt_ad"][t] == osc["dt_ad"]


def test_fp64_many_steps_own_schedules(sph, O):
    cs = tanks()
    got, sc = _batch(sph, cs, "fp64", 40)
    n_adv = []
    for t, c in enumerate(cs):
        o = O.Oracle.from_case(c)
        o.step(40)
        want = _oracle_fields(o, O)
        for k in ("pos", "vel", "rho", "p", "drho", "aprior", "acc"):
            assert rel(got[t][k], want[k]) <= 1e-8, (t, k, rel(got[t][k], want[k]))
        osc = o.scalars()
        assert sc["n_adv"][t] == osc["n_adv"] and sc["n_ac"][t] == osc["n_ac"] == 40
        assert abs(sc["t"][t] - osc["t"]) <= 1e-12 * osc["t"]
        n_adv.append(osc["n_adv"])
    # the tanks are on different schedules (different times after 40 steps)
    assert len(set(np.round(sc["t"], 12))) == len(cs)


def test_mixed_one_step(sph, O):
    cs = tanks()
    got, _ = _batch(sph, cs, "mixed", 1)
    for t, c in enumerate(cs):
        o = O.Oracle.from_case(c)
        o.step(1)
        want = _oracle_fields(o, O)
        g = np.abs(c.gravity).max()
        for k in ("acc", "aprior"):
            err = np.abs(got[t][k] - want[k]).max() / max(np.abs(want[k]).max(), g)
            assert err <= 1e-5, (t, k, err)
        assert rel(got[t]["rho"], want["rho"]) <= 1e-6
        assert np.abs(got[t]["pos"] - want["pos"]).max() <= 1e-6 * c.dp


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_single_tank_contexts(sph, precision):
    cs = tanks()
    got, sc = _batch(sph, cs, precision, 37)
    for t, c in enumerate(cs):
        s = sph.Solver(c, precision=precision)
        s.set_option(sph.SPH_OPT_RECORD_DIAGNOSTICS, 1)
        s.step(37)
        want = s.fields(*FIELDS)
        ssc = s.scalars()
        s.close()
        for k in FIELDS:
            assert np.array_equal(got[t][k], want[k]), (t, k, np.abs(got[t][k] - want[k]).max())
        assert sc["t"][t] == ssc["t"] and sc["n_adv"][t] == ssc["n_adv"]


def test_graph_and_eager_identical(sph):
    cs = tanks()
    a, _ = _batch(sph, cs, "mixed", 12, graph=True)
    b, _ = _batch(sph, cs, "mixed", 12, graph=False)
    for t in range(len(cs)):
        for k in FIELDS:
            assert np.array_equal(a[t][k], b[t][k]), (t, k)


@pytest.mark.parametrize("block", [64, 256])
def test_tile_size_does_not_change_results(sph, block):
    cs = tanks()
    ref, _ = _batch(sph, cs, "mixed", 15)
    b = sph.Batch(cs, precision="mixed")
    b.set_option(sph.SPH_OPT_RECORD_DIAGNOSTICS, 1)
    b.set_option(sph.SPH_OPT_BLOCK, block)
    b.set_option(sph.SPH_OPT_RADIX_BITS, 6)
    b.step(15)
    f = b.fields(*FIELDS)
    for t in range(len(cs)):
        for k in FIELDS:
            assert np.array_equal(f[k][b.offsets[t]:b.offsets[t + 1]], ref[t][k]), (t, k)
    b.close()


def test_empty_tank_and_no_walls(sph, O):
    """A tank without fluid and a tank without walls beside normal tanks."""
    cs = tanks(sizes=(400, 900, 600))
    cs[1].fluid = np.zeros((0, 2))
    cs[2].wall = np.zeros((0, 2))
    b = sph.Batch(cs, precision="fp64")
    b.set_option(sph.SPH_OPT_RECORD_DIAGNOSTICS, 1)
    b.step(8)
    f = b.fields("pos", "vel", "rho")
    for t in (0, 2):
        o = O.Oracle.from_case(cs[t])
        o.step(8)
        a, e = b.offsets[t], b.offsets[t + 1]
        assert rel(f["pos"][a:e], o.field(O.POS)) <= 1e-10
        assert rel(f["rho"][a:e], o.field(O.RHO)) <= 1e-10
    assert b.neighbour_state(1)["cell_begin"].max() == 0
    b.close()


def test_out_of_domain_names_the_tank(sph):
    cs = tanks(sizes=(300, 500, 400))
    cs[2].fluid = cs[2].fluid.copy()
    cs[2].fluid[5, 0] = cs[2].hi[0] + 1.0
    with pytest.raises(sph.SphError) as e:
        b = sph.Batch(cs, precision="mixed")
        b.step(1)
        b.fields("pos")
    assert e.value.code == sph.SPH_E_OUT_OF_DOMAIN and "tank 2" in str(e.value)


def test_kernels_per_step_and_invalid_arguments(sph):
    cs = tanks(sizes=(300, 500))
    b = sph.Batch(cs, precision="mixed")
    k = sph.sph_batch_kernels_per_step(b.b)
    assert 15 <= k <= 40, k  # one launch per stage (+ the sort passes), any tank count
    with pytest.raises(sph.SphError):
        b.set_option(sph.SPH_OPT_BLOCK, 100)
    with pytest.raises(sph.SphError):
        b.neighbour_state(7)
    b.close()
    with pytest.raises(sph.SphError):
        sph.sph_create_batch([cases.batched_tank(300), cases.dam_break_3d(dp=0.05)])


# --------------------------------------------------------------------------
def _config4_tanks():
    """The batched workload at its full size: 256 tanks, fluid counts
    log-uniform in [1 000, 64 000] (seed 4), dp = 0.01, tank k seeded 100 + k."""
    sizes = cases.batched_tank_sizes(256, seed=4)
    return [cases.batched_tank(n, dp=0.01, seed=100 + k) for k, n in enumerate(sizes)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_batch_one_step_against_oracle(sph, O, precision):
    """One step of the whole 256-tank batch; the 4 largest and the 4 smallest
    tanks against the oracle run of that tank alone (every field within 1e-10
    in FP64; accelerations within 1e-5 of max(|a_ref|, g) in mixed)."""
    cs = _config4_tanks()
    got, sc = _batch(sph, cs, precision, 1)
    order = np.argsort([c.n for c in cs])
    picked = list(order[:4]) + list(order[-4:])
    assert cs[picked[0]].n < 1500 and cs[picked[-1]].n > 50000
    worst = {}
    for t in picked:
        o = O.Oracle.from_case(cs[t])
        o.step(1)
        want = _oracle_fields(o, O)
        if precision == "fp64":
            for k in FIELDS:
                assert rel(got[t][k], want[k]) <= 1e-10, (t, k, rel(got[t][k], want[k]))
        else:
            g = np.abs(cs[t].gravity).max()
            for k in ("acc", "aprior"):
                e = np.abs(got[t][k] - want[k]).max() / max(np.abs(want[k]).max(), g)
                worst[k] = max(worst.get(k, 0.0), e)
                assert e <= 1e-5, (t, k, e)
        osc = o.scalars()
        assert sc["dt_ac"][t] == osc["dt_ac"] and sc["dt_ad"][t] == osc["dt_ad"]
    if worst:
        print(f"\n256-tank batch, mixed, first step, 8 tanks: acc {worst['acc']:.2e}, "
              f"aprior {worst['aprior']:.2e}")


def test_full_size_batch_equals_one_tank_contexts(sph):
    """20 steps of the 256-tank mixed batch against one-tank contexts of the
    same 4 largest and 4 smallest tanks: bitwise equal (each tank on its own
    schedule, the same kernels walking each tank's tiles)."""
    cs = _config4_tanks()
    got, sc = _batch(sph, cs, "mixed", 20)
    order = np.argsort([c.n for c in cs])
    for t in list(order[:4]) + list(order[-4:]):
        s = sph.Solver(cs[t], precision="mixed")
        s.set_option(sph.SPH_OPT_RECORD_DIAGNOSTICS, 1)
        s.step(20)
        one = s.fields(*FIELDS)
        osc = s.scalars()
        s.close()
        for k in FIELDS:
            assert np.array_equal(got[t][k], one[k]), (t, k)
        assert sc["n_adv"][t] == osc["n_adv"] and sc["t"][t] == osc["t"]
