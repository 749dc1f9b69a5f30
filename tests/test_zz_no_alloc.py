"""The allocation-free cell sort (sph_cell_sort_noalloc), called through the
C ABI, against the oracle's sort of the same positions (keys, permutation and
cell offsets; integer results, so they must match exactly) and against the
library's own context sort (sph_set_particles bins and sorts the same
positions, sph_debug_neighbour_state returns its state).

The cases cover every layout of the radix ping-pong in the shared scratch:
one pass (256 cells or fewer), two passes, three passes (more than 65 536
cells), the largest accepted count (SPH_NOALLOC_MAX_PARTICLES particles) and
an empty input (offsets only).  They run as consecutive calls, each reusing
the scratch the previous call left behind.  This file is collected last on
purpose."""
import numpy as np
import pytest

from paper_2603_11868_gb300 import cases

pytestmark = pytest.mark.gpu


def _cases():
    return [
        ("3d_two_pass", cases.dam_break_3d(dp=0.02, seed=1)),          # 10 200, ~7.7k cells
        ("2d_two_pass", cases.random_cloud(2, 300_000, seed=9, dp=0.004)),  # ~13.5k cells
        ("2d_three_pass", cases.random_cloud(2, 200_000, seed=5, dp=0.001)),  # ~213k cells
        ("3d_one_pass", cases.random_cloud(3, 5000, seed=6, dp=0.1)),  # 125 cells
        ("3d_max_n", cases.uniform_cube(n=1 << 20, seed=8)),           # ~79k cells, 3 passes
    ]


def _noalloc(sph, case, dev, stream, ncell):
    import torch
    n = case.n
    soa = torch.from_numpy(np.ascontiguousarray(case.fluid.T)).to(dev)
    keys = torch.full((max(n, 1),), -1, dtype=torch.int32, device=dev)
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device=dev)
    cb = torch.full((ncell + 1,), -1, dtype=torch.int32, device=dev)
    z = soa[2].data_ptr() if case.dim == 3 else None
    rc = sph.sph_cell_sort_noalloc(case.dim, case.lo, case.hi, 2.0 * case.h,
                                   soa[0].data_ptr(), soa[1].data_ptr(), z, n,
                                   keys.data_ptr(), perm.data_ptr(), cb.data_ptr(), stream)
    assert rc == sph.SPH_OK
    torch.cuda.synchronize()
    view = lambda t: t.cpu().numpy().view(np.uint32)  # noqa: E731
    return view(keys)[:n], view(perm)[:n], view(cb)


def test_noalloc_sort_matches_oracle_and_context_sort():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from oracle import oracle as O
    from paper_2603_11868_gb300 import build, sph
    build.build()
    sph.load()
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for name, case in _cases():
        o = O.Oracle.from_case(case)
        want = o.neighbour_state()
        assert np.array_equal(want["perm"], want["ids"])  # a first sort from user order
        got = _noalloc(sph, case, dev, stream, o.ncell)
        for g, k in zip(got, ("keys", "perm", "cell_begin")):
            assert np.array_equal(g, want[k]), (name, k)
        if name in ("3d_two_pass", "2d_three_pass"):
            ref = sph.Solver(case, precision="mixed")
            ctx = ref.neighbour_state()
            ref.close()
            for g, k in zip(got, ("keys", "perm", "cell_begin")):
                assert np.array_equal(g, ctx[k]), (name, k)


def test_noalloc_empty_input_gives_zero_offsets():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from paper_2603_11868_gb300 import sph
    sph.load()
    dev = torch.device("cuda")
    ncell = 11 * 11 * 11
    keys = torch.full((1,), -1, dtype=torch.int32, device=dev)
    perm = torch.full((1,), -1, dtype=torch.int32, device=dev)
    cb = torch.full((ncell + 1,), -1, dtype=torch.int32, device=dev)
    rc = sph.sph_cell_sort_noalloc(3, (0, 0, 0), (1.1, 1.1, 1.1), 0.1, None, None, None, 0,
                                   keys.data_ptr(), perm.data_ptr(), cb.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == sph.SPH_OK
    torch.cuda.synchronize()
    assert np.all(cb.cpu().numpy() == 0)
    assert int(keys.item()) == -1 and int(perm.item()) == -1  # nothing written


def test_noalloc_rejects_too_many_particles():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from paper_2603_11868_gb300 import sph
    sph.load()
    n = sph.SPH_NOALLOC_MAX_PARTICLES + 1
    rc = sph.sph_cell_sort_noalloc(3, (0, 0, 0), (1, 1, 1), 0.1, 1, 1, 1, n, 1, 1, 1, 0)
    assert rc == sph.SPH_E_INVALID
