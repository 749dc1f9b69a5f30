"""Standalone neighbour search (sph_nsearch_*) against the oracle: keys,
permutation and cell offsets bit-exact, the density pass's kernel sums within
the tolerance of the position type (1e-12 relative in double, 1e-5 in float,
where the oracle sees the float-rounded positions)."""
import numpy as np
import pytest

from paper_2603_11868_gb300 import cases

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("n", [1, 4097, 60000])
def test_nsearch_matches_oracle(n, fp32):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from oracle import oracle as O
    from paper_2603_11868_gb300 import build, sph
    build.build()
    case = cases.uniform_cube(n=n, seed=11, neighbours=57.0) if n > 1 else \
        cases.uniform_cube(n=1, seed=11)
    pos = case.fluid.astype(np.float32).astype(np.float64) if fp32 else case.fluid
    dt = torch.float32 if fp32 else torch.float64
    dev = [torch.tensor(np.ascontiguousarray(pos[:, k]), dtype=dt, device="cuda")
           for k in range(3)]
    ns = sph.NeighbourSearch(3, case.lo, case.hi, case.h, fp32=fp32)
    ms = ns.run(*dev)
    assert all(v >= 0 for v in ms.values())
    got = ns.results()
    o = O.Oracle(3, case.lo, case.hi, case.dp, case.h, 1.0, 10.0, 0.0, 1.0, (0, 0, 0))
    o.set_fluid(pos)
    want = o.neighbour_state()
    for k in ("keys", "perm", "cell_begin"):
        assert np.array_equal(got[k], want[k]), k
    o.density_summation()
    sig_user = o.field(O.SIGMA)
    want_sig = sig_user[got["perm"]]
    err = np.abs(got["sigma"] - want_sig).max() / np.abs(want_sig).max()
    assert err <= (1e-5 if fp32 else 1e-12), err
    ns.close()


@pytest.mark.parametrize("fp32", [False, True])
def test_keys_on_and_next_to_cell_faces(fp32):
    """Coordinates on cell faces lo + k cs and a few ulps to either side, with
    a grid origin that makes x - lo inexact: the cell index must be the floor of
    the correctly rounded double quotient (the key kernel's float shortcut
    must hand every such coordinate to the exact division)."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from oracle import oracle as O
    from paper_2603_11868_gb300 import build, sph
    build.build()
    h = 0.0123456789
    cs = 2.0 * h
    lo = np.array([-0.1037, 0.0513, 0.3001])
    hi = lo + 37.3 * cs
    rng = np.random.default_rng(5)
    faces = lo[None, :] + np.arange(0, 37)[:, None] * cs
    pts = []
    for d in (-3, -2, -1, 0, 1, 2, 3):
        f = faces.copy()
        for _ in range(abs(d)):
            f = np.nextafter(f, np.inf if d > 0 else -np.inf)
        pts.append(f)
    pts = np.concatenate(pts)
    # mix the axes so that every point has face coordinates on all three
    pts = np.stack([rng.permutation(pts[:, k]) for k in range(3)], 1)
    pts = np.clip(pts, lo, hi - 1e-9)
    if fp32:
        pts = pts.astype(np.float32).astype(np.float64)
    dt = torch.float32 if fp32 else torch.float64
    dev = [torch.tensor(np.ascontiguousarray(pts[:, k]), dtype=dt, device="cuda")
           for k in range(3)]
    ns = sph.NeighbourSearch(3, lo, hi, h, fp32=fp32)
    ns.run(*dev, timed=False)
    got = ns.results()
    o = O.Oracle(3, lo, hi, 0.01, h, 1.0, 10.0, 0.0, 1.0, (0, 0, 0))
    o.set_fluid(pts)
    want = o.neighbour_state()
    for k in ("keys", "perm", "cell_begin"):
        assert np.array_equal(got[k], want[k]), k
    # the set really straddles faces: cells on both sides of many faces
    assert len(np.unique(want["keys"])) > 100
    ns.close()


@pytest.mark.parametrize("fp32", [True, False])
def test_nsearch_full_size_2_24(fp32):
    """The neighbour-search workload at its full size: 2^24 particles uniform
    in the unit cube (seed 3), 57 neighbours within 2h on average.  Keys,
    permutation and cell offsets bit-exact against the oracle's sort of the
    same positions; the density pass's kernel sums on 5000 sampled particles
    against the oracle's (1e-5 relative with float positions, 1e-12 with
    double)."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from oracle import oracle as O
    from paper_2603_11868_gb300 import build, sph
    build.build()
    case = cases.uniform_cube(n=1 << 24, seed=3, neighbours=57.0)
    pos = case.fluid.astype(np.float32).astype(np.float64) if fp32 else case.fluid
    dt = torch.float32 if fp32 else torch.float64
    dev = [torch.tensor(np.ascontiguousarray(pos[:, k]), dtype=dt, device="cuda")
           for k in range(3)]
    ns = sph.NeighbourSearch(3, case.lo, case.hi, case.h, fp32=fp32)
    ns.run(*dev, timed=False)
    got = ns.results()
    ns.close()
    del dev
    o = O.Oracle(3, case.lo, case.hi, case.dp, case.h, 1.0, 10.0, 0.0, 1.0, (0, 0, 0))
    o.set_fluid(pos)
    want = o.neighbour_state()
    for k in ("keys", "perm", "cell_begin"):
        assert np.array_equal(got[k], want[k]), k
    ids = np.random.default_rng(7).choice(case.n, 5000, replace=False).astype(np.uint32)
    slot = np.empty(case.n, np.int64)
    slot[got["perm"]] = np.arange(case.n)
    want_sig = o.sample_sigma(ids)
    err = np.abs(got["sigma"][slot[ids]] - want_sig).max() / np.abs(want_sig).max()
    print(f"\nneighbour search 2^24 ({'float' if fp32 else 'double'} positions): "
          f"sampled sigma error {err:.2e}")
    assert err <= (1e-5 if fp32 else 1e-12), err
