"""Allocation failure, injected on the host: an allocator that returns NULL
after a given number of allocations.  Whichever call runs out (creation,
walls, fluid, a batch) fails with SPH_E_OOM, the context can still be
destroyed, and every allocation it made is freed.  Nothing faults a GPU: the
library only ever sees a NULL pointer from the callback."""
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


def counting_allocator(sph, limit=None):
    class Counting(sph.TorchAllocator):
        def __init__(self):
            super().__init__()
            self.n_alloc = self.n_free = 0
            self.live = set()

        def _on_alloc(self, nbytes, stream, user):
            if limit is not None and self.n_alloc >= limit:
                return None
            p = super()._on_alloc(nbytes, stream, user)
            if p:
                self.n_alloc += 1
                self.live.add(int(p))
            return p

        def _on_free(self, ptr, nbytes, stream, user):
            self.n_free += 1
            self.live.discard(int(ptr))
            super()._on_free(ptr, nbytes, stream, user)

    return Counting()


def _single(sph, case, alloc):
    ctx = sph.sph_create(case.dim, case.lo, case.hi, case.dp, case.h, case.rho0, case.c0,
                         case.mu, case.U_ref, case.gravity, sph.SPH_MIXED, alloc.struct, 0)
    try:
        sph.sph_set_particles(ctx, sph.SPH_WALL, case.wall)
        sph.sph_set_particles(ctx, sph.SPH_FLUID, case.fluid)
        sph.sph_step(ctx, 3)
        sph.sph_synchronize(ctx, 0.0)
    finally:
        sph.sph_destroy(ctx)


def test_every_allocation_failure_is_an_oom_and_leaks_nothing(sph):
    case = cases.dam_break_2d(dp=0.05)
    full = counting_allocator(sph)
    _single(sph, case, full)
    total = full.n_alloc
    assert total > 5 and not full.live and full.n_free == total
    # fail at every allocation in turn: creation, wall and fluid buffers
    for limit in range(total):
        a = counting_allocator(sph, limit)
        with pytest.raises(sph.SphError) as e:
            _single(sph, case, a)
        assert e.value.code == sph.SPH_E_OOM, (limit, e.value)
        assert not a.live, (limit, len(a.live))


def test_batch_allocation_failure_is_an_oom(sph):
    import numpy as np
    tanks = [cases.batched_tank(n, dp=0.02, seed=90 + k) for k, n in enumerate((300, 700))]
    walls = [t.wall for t in tanks]
    for limit in (0, 3, 8, 12):
        a = counting_allocator(sph, limit)
        with pytest.raises(sph.SphError) as e:
            bb = sph.sph_create_batch(tanks, sph.SPH_MIXED, a.struct, 0)
            try:
                sph.sph_batch_set_particles(bb, sph.SPH_WALL, [len(w) for w in walls],
                                            np.concatenate(walls))
                sph.sph_batch_set_particles(bb, sph.SPH_FLUID, [t.n for t in tanks],
                                            np.concatenate([t.fluid for t in tanks]))
            finally:
                sph.sph_batch_destroy(bb)
        assert e.value.code == sph.SPH_E_OOM, (limit, e.value)
        assert not a.live, limit


def test_misaligned_allocator_block_is_refused(sph):
    """Device blocks must be 256-byte aligned (the kernels use 16- and
    32-byte vector loads on them): a block 16 bytes off is handed back to the
    allocator's free and the call fails with SPH_E_OOM, leaking nothing."""
    class Misaligned(sph.TorchAllocator):
        def __init__(self):
            super().__init__()
            self.base = {}
            self.n_alloc = 0

        def _on_alloc(self, nbytes, stream, user):
            p = super()._on_alloc(nbytes + 256, stream, user)
            if not p:
                return None
            self.n_alloc += 1
            q = int(p) + 16
            self.base[q] = int(p)
            return q

        def _on_free(self, ptr, nbytes, stream, user):
            super()._on_free(self.base.pop(int(ptr)), nbytes + 256, stream, user)

    case = cases.dam_break_2d(dp=0.05)
    a = Misaligned()
    with pytest.raises(sph.SphError) as e:
        _single(sph, case, a)
    assert e.value.code == sph.SPH_E_OOM
    assert a.n_alloc >= 1 and not a.base
