"""The seeded input generators: wall lattices without gaps and fluid inside
the tank, whatever the ratio of tank length to dp."""
import numpy as np
import pytest

from paper_2603_11868_gb300 import cases


def _gaps(coords, dp):
    u = np.unique(np.round(coords / (0.01 * dp)).astype(np.int64)) * (0.01 * dp)
    return np.diff(u)


@pytest.mark.parametrize("make", [
    lambda: cases.dam_break_2d(),                     # 5.366 / 0.025 = 214.64
    lambda: cases.dam_break_3d(dp=0.02),              # 0.67 / 0.02 = 33.5
    lambda: cases.dam_break_3d(dp=0.05),              # 0.67 / 0.05 = 13.4
    lambda: cases.batched_tank(700, dp=0.02, seed=1),  # side 2.683 W
    lambda: cases.dam_break_3d(),                     # whole numbers of dp
])
def test_floor_wall_lattice_has_no_gap(make):
    c = make()
    dim, dp = c.dim, c.dp
    up = dim - 1
    floor = c.wall[c.wall[:, up] < 0]
    top_layer = floor[np.isclose(floor[:, up], floor[:, up].max())]
    for k in range(dim - 1):
        g = _gaps(top_layer[:, k], dp)
        assert np.allclose(g, dp, rtol=0, atol=1e-9), (k, g.min(), g.max())
    # every fluid particle starts inside the tank the walls enclose
    inner_hi = np.array([c.wall[c.wall[:, k] > c.fluid[:, k].max(), k].min()
                         for k in range(dim - 1)])
    assert (c.fluid[:, :dim - 1] <= inner_hi - 0.5 * dp + 1e-9 + 0.01 * dp).all()
    assert (c.fluid > 0).all()


def test_lattice_length_keeps_whole_lengths_exact():
    assert cases.lattice_length(0.67, 0.01) == 0.67
    assert cases.lattice_length(1.6, 0.0025) == 1.6
    assert cases.lattice_length(0.67, 0.02) == pytest.approx(0.68, abs=1e-15)
    assert cases.lattice_length(5.366, 0.025) == pytest.approx(5.375, abs=1e-15)
    assert cases.lattice_length(0.001, 0.02) == pytest.approx(0.02, abs=1e-15)
