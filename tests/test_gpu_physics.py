"""Physics checks run directly on the GPU path (mixed and FP64), not through
the oracle:

- the resting hydrostatic column: time-averaged over the last 10 % of
  t sqrt(g/H) = 20, |p - rho0 g (H - y)| <= 1 % of rho0 g H below the top
  three layers, at h = 1.5 dp, the oracle's own bar;
- a long mixed-precision 3D dam break (2 000 acoustic steps, t > 1 s, past
  the impact on the far wall and the run-up): finite state, no particle
  through a wall (every particle inside the tank the walls enclose), kinetic
  energy bounded by the potential energy released, densities near rho0.
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


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_hydrostatic_column(sph, precision):
    c = cases.hydrostatic_2d(dp=0.05)
    c.h = 1.5 * c.dp
    s = sph.Solver(c, precision=precision)
    H, T = c.meta["H"], 20.0
    ps, ys = [], []
    while s.scalars()["t"] < T:
        s.step(50)
        if s.scalars()["t"] > 0.9 * T:
            f = s.fields("p", "pos")
            ps.append(f["p"])
            ys.append(f["pos"][:, 1])
    s.close()
    p, y = np.mean(ps, 0), np.mean(ys, 0)
    mask = y < H - 3 * c.dp
    err = np.abs(p - c.rho0 * 1.0 * (H - y))[mask]
    assert err.max() <= 0.01 * c.rho0 * 1.0 * H, err.max() / (c.rho0 * H)


@pytest.mark.parametrize("precision", ["mixed"])
def test_hydrostatic_column_at_configured_h(sph, precision):
    """The same column at the configurations' h = 1.3 dp, reported rather
    than held to 1 %: the kernel's lattice gradient consistency there is
    kappa = 0.974, which alone tilts the pressure slope by about 2.6 %, so the
    column settles a few per cent off rho0 g (H - y).  The bound below only
    guards that figure against regressions; the 1 % pin is the h = 1.5 dp
    run above."""
    c = cases.hydrostatic_2d(dp=0.05)
    assert abs(c.h / c.dp - 1.3) < 1e-12
    s = sph.Solver(c, precision=precision)
    H, T = c.meta["H"], 20.0
    ps, ys = [], []
    while s.scalars()["t"] < T:
        s.step(50)
        if s.scalars()["t"] > 0.9 * T:
            f = s.fields("p", "pos")
            ps.append(f["p"])
            ys.append(f["pos"][:, 1])
    s.close()
    p, y = np.mean(ps, 0), np.mean(ys, 0)
    mask = y < H - 3 * c.dp
    err = np.abs(p - c.rho0 * 1.0 * (H - y))[mask] / (c.rho0 * 1.0 * H)
    bottom = np.abs(p[np.argmin(y)] / (c.rho0 * (H - y.min())) - 1.0)
    print(f"\nhydrostatic column at h = 1.3 dp ({precision}): max |p - rho0 g (H - y)| = "
          f"{err.max():.2%} of rho0 g H, bottom-particle pressure off by {bottom:.2%}")
    assert err.max() <= 0.06


def test_long_dam_break_stays_physical(sph):
    c = cases.dam_break_3d(dp=0.02, seed=3)
    s = sph.Solver(c, precision="mixed")
    g = abs(c.gravity[2])
    m = c.rho0 * c.dp ** 3
    z0 = c.fluid[:, 2].copy()
    s.step(2000)
    f = s.fields("pos", "vel", "rho")
    sc = s.scalars()
    s.close()
    pos, vel, rho = f["pos"], f["vel"], f["rho"]
    assert np.isfinite(pos).all() and np.isfinite(vel).all() and np.isfinite(rho).all()
    assert sc["n_ac"] == 2000 and sc["t"] > 1.0
    tank = np.array([cases.lattice_length(L, c.dp) for L in c.meta["tank"]])
    assert (pos[:, :2] > 0).all() and (pos[:, :2] < tank[:2]).all()
    assert (pos[:, 2] > 0).all()
    # kinetic energy cannot exceed the potential energy released (viscosity and
    # the Riemann dissipation only remove energy)
    ke = 0.5 * m * (vel ** 2).sum()
    released = m * g * (z0.sum() - pos[:, 2].sum())
    assert 0 < ke <= released * 1.02, (ke, released)
    # weakly compressible (c0 = 10 sqrt(2 g H)): densities within 10 % of rho0
    assert np.abs(rho / c.rho0 - 1).max() < 0.10
