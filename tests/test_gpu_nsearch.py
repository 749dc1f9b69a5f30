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
