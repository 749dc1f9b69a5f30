"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point include/sph.h declares.  No compute call is made here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2603_11868_gb300 import build, sph
    build.build()
    return sph.load()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(sph_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sph_create", "sph_set_particles", "sph_step", "sph_get_fields"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_export():
    from paper_2603_11868_gb300 import sph
    assert set(sph.EXPORTS) == set(declared_functions())


def test_library_is_built_for_sm_103a(lib):
    from paper_2603_11868_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.getsize(build.LIB) > 100_000


def test_argument_validation_needs_no_device(lib):
    """Invalid arguments are rejected before any CUDA call."""
    from paper_2603_11868_gb300 import sph
    dom = sph.sph_domain(4, (C.c_double * 3)(0, 0, 0), (C.c_double * 3)(1, 1, 1))
    mat = sph.sph_material(1.0, 10.0, 0.0, 1.0)
    g = (C.c_double * 3)(0, 0, 0)
    out = C.c_void_p()
    assert lib.sph_create(C.byref(dom), 0.01, 0.013, C.byref(mat), g, 1, None, None,
                          C.byref(out)) == sph.SPH_E_INVALID
    dom.dim = 3
    assert lib.sph_create(C.byref(dom), -1.0, 0.013, C.byref(mat), g, 1, None, None,
                          C.byref(out)) == sph.SPH_E_INVALID
    dom.hi[0] = -1.0
    assert lib.sph_create(C.byref(dom), 0.01, 0.013, C.byref(mat), g, 1, None, None,
                          C.byref(out)) == sph.SPH_E_INVALID
    dom.hi[0] = 1.0
    assert lib.sph_create(C.byref(dom), 0.01, 0.013, C.byref(mat), g, 7, None, None,
                          C.byref(out)) == sph.SPH_E_INVALID
    # too many cells for 32-bit keys
    assert lib.sph_create(C.byref(dom), 1e-4, 1e-5, C.byref(mat), g, 1, None, None,
                          C.byref(out)) == sph.SPH_E_INVALID
    assert lib.sph_step(None, 1) == sph.SPH_E_INVALID
    assert lib.sph_destroy(None) is None


def test_product_path_does_not_import_the_oracle():
    """The package never imports oracle/ (the checker is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2603_11868_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "sph_oracle" not in text, f


def test_batch_argument_validation_needs_no_device(lib):
    """sph_create_batch rejects bad batches before any CUDA call."""
    from paper_2603_11868_gb300 import sph

    def tank(dim=2, dp=0.01, hi=1.0):
        return sph.sph_tank(sph.sph_domain(dim, (C.c_double * 3)(0, 0, 0),
                                           (C.c_double * 3)(hi, hi, hi)),
                            dp, 1.3 * dp, sph.sph_material(1.0, 10.0, 0.0, 1.0),
                            (C.c_double * 3)(0, -1, 0))

    out = C.c_void_p()
    two = (sph.sph_tank * 2)(tank(), tank())
    assert lib.sph_create_batch(0, two, 1, None, None, C.byref(out)) == sph.SPH_E_INVALID
    assert lib.sph_create_batch(sph.SPH_MAX_TANKS + 1, two, 1, None, None,
                                C.byref(out)) == sph.SPH_E_INVALID
    assert lib.sph_create_batch(2, None, 1, None, None, C.byref(out)) == sph.SPH_E_INVALID
    assert lib.sph_create_batch(2, two, 5, None, None, C.byref(out)) == sph.SPH_E_INVALID
    mixed_dims = (sph.sph_tank * 2)(tank(), tank(dim=3))
    assert lib.sph_create_batch(2, mixed_dims, 1, None, None,
                                C.byref(out)) == sph.SPH_E_INVALID
    bad_dp = (sph.sph_tank * 2)(tank(), tank(dp=-0.01))
    assert lib.sph_create_batch(2, bad_dp, 1, None, None, C.byref(out)) == sph.SPH_E_INVALID
    # 2^31 or more cells over the batch (each tank alone is fine)
    big = (sph.sph_tank * 40)(*[tank(dp=1e-4, hi=2.6) for _ in range(40)])  # 1e8 cells each
    assert lib.sph_create_batch(40, big, 1, None, None, C.byref(out)) == sph.SPH_E_INVALID
    assert out.value is None
    assert lib.sph_batch_step(None, 1) == sph.SPH_E_INVALID
    assert lib.sph_batch_tank_count(None) == 0
    assert lib.sph_batch_destroy(None) is None


def test_batches_refuse_translating_walls():
    from paper_2603_11868_gb300 import cases, sph
    with pytest.raises(ValueError):
        sph.Batch([cases.piston_channel_2d()])


@pytest.mark.parametrize("case", ["tiny_edge", "infinite_extent", "nan_extent"])
def test_grid_extent_checked_before_the_cast(lib, case):
    """A cell count that is not a finite number of at most 2^30 cells per axis
    (a tiny cell edge, an infinite or NaN extent) is refused with
    SPH_E_INVALID by every entry point that builds a cell grid, before any
    CUDA call: the quotient is range-checked as a double, never cast first."""
    from paper_2603_11868_gb300 import sph
    hi = {"tiny_edge": 1.0, "infinite_extent": float("inf"), "nan_extent": float("nan")}[case]
    h = 1e-300 if case == "tiny_edge" else 0.013
    dom = sph.sph_domain(3, (C.c_double * 3)(0, 0, 0), (C.c_double * 3)(hi, 1, 1))
    mat = sph.sph_material(1.0, 10.0, 0.0, 1.0)
    g = (C.c_double * 3)(0, 0, 0)
    out = C.c_void_p()
    assert lib.sph_create(C.byref(dom), 0.01, h, C.byref(mat), g, 1, None, None,
                          C.byref(out)) == sph.SPH_E_INVALID
    assert out.value is None
    one = C.c_uint32()
    assert lib.sph_cell_sort_noalloc(C.byref(dom), 2.0 * h, None, None, None, 0,
                                     C.byref(one), C.byref(one), C.byref(one),
                                     None) == sph.SPH_E_INVALID
    ns = C.c_void_p()
    assert lib.sph_nsearch_create(C.byref(dom), h, 1, None, None,
                                  C.byref(ns)) == sph.SPH_E_INVALID
    assert ns.value is None
    tank = sph.sph_tank(dom, 0.01, h, mat, (C.c_double * 3)(0, 0, -1))
    tanks = (sph.sph_tank * 1)(tank)
    assert lib.sph_create_batch(1, tanks, 1, None, None, C.byref(out)) == sph.SPH_E_INVALID
    assert out.value is None
