"""Pins of the oracle's sampled evaluations (osph_sample_sigma,
osph_sample_first_step_acc).  They are the checker of the full-size GPU
parity tests (5.1 M and beyond 2^25 fluid particles), where a whole oracle
step would take too long, so they must equal the oracle's own first step.

Both evaluate the same sums as osph_step(1) in the same order (the first
rebuild of a fresh state keeps the storage order, the summation visits the
same cells and indices, and the first half-step from rest moves nothing), so
the comparison is bitwise, not a tolerance:
  sample_sigma(ids)           == SIGMA after osph_step(1) at ids
  sample_first_step_acc(ids)  == ACC   after osph_step(1) at ids
A mistake in either function (a neighbour not marked for the density pass,
the density taken before the free-surface clamp, the state's density passed
in place of the summed one) changes these bits, mostly by orders of
magnitude; tests/test_pins_mutations.py plants such mistakes.
"""
import numpy as np
import pytest

from paper_2603_11868_gb300 import cases


def _check(o_mod, case, ids):
    fresh = o_mod.Oracle.from_case(case)
    sig = fresh.sample_sigma(ids)
    acc = fresh.sample_first_step_acc(ids)
    ref = o_mod.Oracle.from_case(case)
    ref.step(1)
    want_sig = ref.field(o_mod.SIGMA)[ids]
    want_acc = ref.field(o_mod.ACC)[ids]
    assert np.all(np.isfinite(want_acc))
    assert np.array_equal(sig, want_sig), np.abs(sig - want_sig).max()
    assert np.array_equal(acc, want_acc), np.abs(acc - want_acc).max()
    return want_sig, want_acc


def _surface_and_interior(case, rng, m):
    """Sampled user ids: every particle of the top layer and next to a wall
    (where the free-surface clamp and the mirrored wall state act), plus a
    random interior draw."""
    x = case.fluid
    up = case.dim - 1
    top = np.nonzero(x[:, up] > x[:, up].max() - 1.5 * case.dp)[0]
    low = np.nonzero(x[:, up] < x[:, up].min() + 1.5 * case.dp)[0]
    side = np.nonzero(x[:, 0] < x[:, 0].min() + 1.5 * case.dp)[0]
    rest = rng.choice(case.n, size=m, replace=False)
    return np.unique(np.concatenate([top, low, side, rest])).astype(np.uint32)


def test_sampled_first_step_equals_step_2d_walls_jitter(oracle_mod):
    case = cases.dam_break_2d()
    ids = np.arange(case.n, dtype=np.uint32)  # every fluid particle
    sig, acc = _check(oracle_mod, case, ids)
    # the sample covers both branches of the clamp and the walls' push
    ratio = sig / oracle_mod.sigma0(2, case.dp, case.h)
    assert ratio.min() < 0.8 and ratio.max() > 1.0
    assert np.abs(acc).max() > abs(min(case.gravity))


def test_sampled_first_step_equals_step_3d_config1(oracle_mod):
    case = cases.dam_break_3d()
    rng = np.random.default_rng(11)
    ids = _surface_and_interior(case, rng, 3000)
    assert len(ids) > 5000
    sig, acc = _check(oracle_mod, case, ids)
    ratio = sig / oracle_mod.sigma0(3, case.dp, case.h)
    assert ratio.min() < 0.8 and ratio.max() > 1.0


@pytest.mark.parametrize("seed", [0, 1])
def test_sampled_first_step_equals_step_cloud(oracle_mod, seed):
    """A disordered cloud with random densities under gravity: neighbour
    counts and densities vary from particle to particle (no lattice
    symmetry), every particle sampled in a shuffled order with repeats."""
    case = cases.random_cloud(3, 1500, seed=seed, dp=0.08, rho_spread=0.05,
                              gravity=(0.0, 0.0, -1.0))
    rng = np.random.default_rng(seed)
    ids = rng.permutation(np.concatenate([np.arange(case.n), np.arange(0, case.n, 7)]))
    _check(oracle_mod, case, ids.astype(np.uint32))
