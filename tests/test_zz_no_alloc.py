"""The allocation-free cell sort (sph_cell_sort_noalloc), called through the
C ABI, against the existing path: a context's fluid upload (sph_set_particles)
bins and sorts the same positions, and sph_debug_neighbour_state returns its
keys, permutation and cell offsets.  Integer results, so they must match
exactly, on two calls in a row (the second reuses the shared scratch the first
one left behind).  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2603_11868_gb300 import cases

pytestmark = pytest.mark.gpu


def test_noalloc_sort_matches_context_sort():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from paper_2603_11868_gb300 import build, sph
    build.build()
    sph.load()
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream().cuda_stream
    runs = [cases.dam_break_3d(dp=0.02, seed=1),                      # 10 200 particles
            cases.random_cloud(2, 300_000, seed=9, dp=0.004)]          # second call, larger
    for case in runs:
        ref = sph.Solver(case, precision="mixed")
        want = ref.neighbour_state()
        ncell = ref.ncell
        ref.close()
        n = case.n
        soa = torch.from_numpy(np.ascontiguousarray(case.fluid.T)).to(dev)
        keys = torch.full((n,), -1, dtype=torch.int32, device=dev)
        perm = torch.full((n,), -1, dtype=torch.int32, device=dev)
        cb = torch.full((ncell + 1,), -1, dtype=torch.int32, device=dev)
        z = soa[2].data_ptr() if case.dim == 3 else None
        rc = sph.sph_cell_sort_noalloc(case.dim, case.lo, case.hi, 2.0 * case.h,
                                       soa[0].data_ptr(), soa[1].data_ptr(), z, n,
                                       keys.data_ptr(), perm.data_ptr(), cb.data_ptr(), stream)
        assert rc == sph.SPH_OK
        torch.cuda.synchronize()
        assert np.array_equal(keys.cpu().numpy().view(np.uint32), want["keys"])
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), want["perm"])
        assert np.array_equal(cb.cpu().numpy().view(np.uint32), want["cell_begin"])


def test_noalloc_rejects_too_many_particles():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    from paper_2603_11868_gb300 import sph
    sph.load()
    n = sph.SPH_NOALLOC_MAX_PARTICLES + 1
    rc = sph.sph_cell_sort_noalloc(3, (0, 0, 0), (1, 1, 1), 0.1, 1, 1, 1, n, 1, 1, 1, 0)
    assert rc == sph.SPH_E_INVALID
