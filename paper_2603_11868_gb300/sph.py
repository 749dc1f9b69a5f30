"""Python binding of libsph.so (include/sph.h).

Argument marshalling only: every step of the SPH path runs in the library's
CUDA kernels.  The functions keep the C names (sph_create, sph_set_particles,
sph_step, sph_get_fields, ...); ``Solver`` wraps one context for convenience.

PyTorch is used for plumbing only: device memory comes from its caching
allocator (through the allocator callbacks of the C ABI) and work is queued on
its current CUDA stream.  There is no CPU path: if the library or a CUDA
device is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsph.so")

# enums of include/sph.h
SPH_FP64, SPH_MIXED = 0, 1
SPH_FLUID, SPH_WALL = 0, 1
SPH_OK, SPH_E_INVALID, SPH_E_OOM, SPH_E_CUDA, SPH_E_OUT_OF_DOMAIN, SPH_E_NONFINITE, \
    SPH_E_TIMEOUT, SPH_E_STATE = range(8)
SPH_F_POS, SPH_F_VEL, SPH_F_RHO, SPH_F_P, SPH_F_DRHO, SPH_F_ACC, SPH_F_APRIOR, SPH_F_SIGMA = \
    (1 << k for k in range(8))
SPH_OPT_RECORD_DIAGNOSTICS, SPH_OPT_USE_GRAPH, SPH_OPT_BLOCK, SPH_OPT_RADIX_BITS = 1, 2, 3, 4
SPH_OPT_NEIGHBOUR_LIST = 5
SPH_OPT_DENSITY_RIEMANN, SPH_OPT_REINIT_BLENDED, SPH_OPT_TRANSPORT_CORRECTION = 6, 7, 8
_VECTOR_FIELDS = (SPH_F_POS, SPH_F_VEL, SPH_F_ACC, SPH_F_APRIOR)
FIELD_NAMES = {"pos": SPH_F_POS, "vel": SPH_F_VEL, "rho": SPH_F_RHO, "p": SPH_F_P,
               "drho": SPH_F_DRHO, "acc": SPH_F_ACC, "aprior": SPH_F_APRIOR,
               "sigma": SPH_F_SIGMA}
STATUS_NAMES = {0: "SPH_OK", 1: "SPH_E_INVALID", 2: "SPH_E_OOM", 3: "SPH_E_CUDA",
                4: "SPH_E_OUT_OF_DOMAIN", 5: "SPH_E_NONFINITE", 6: "SPH_E_TIMEOUT",
                7: "SPH_E_STATE"}

# every symbol include/sph.h declares
EXPORTS = ("sph_create", "sph_set_particles", "sph_step", "sph_get_fields", "sph_get_scalars",
           "sph_count", "sph_cell_count", "sph_debug_neighbour_state",
           "sph_debug_neighbour_stats", "sph_set_option", "sph_synchronize", "sph_last_error",
           "sph_destroy", "sph_profile_stages", "sph_kernels_per_step",
           "sph_cell_sort_noalloc", "sph_nsearch_create", "sph_nsearch_run",
           "sph_nsearch_results", "sph_nsearch_cell_count", "sph_nsearch_destroy",
           "sph_create_batch", "sph_batch_set_particles", "sph_batch_step",
           "sph_batch_get_fields", "sph_batch_get_scalars", "sph_batch_debug_neighbour_state",
           "sph_batch_count", "sph_batch_tank_count", "sph_batch_cell_count",
           "sph_batch_profile_stages", "sph_batch_kernels_per_step", "sph_batch_set_option",
           "sph_batch_synchronize", "sph_batch_last_error", "sph_batch_destroy",
           "sph_autotune", "sph_batch_autotune", "sph_debug_list_lengths",
           "sph_set_wall_translation", "sph_set_wall_motion", "sph_checkpoint_bytes",
           "sph_checkpoint_save",
           "sph_checkpoint_load", "sph_get_state_range", "sph_put_state_range",
           "sph_get_schedule", "sph_set_schedule", "sph_owned_vmax2", "sph_set_vmax2",
           "sph_get_state_rows_device", "sph_put_state_rows_device", "sph_owned_vmax2_device",
           "sph_set_vmax2_device")
SPH_MAX_TANKS = 1024
SPH_NOALLOC_MAX_PARTICLES = 1 << 20
STAGE_NAMES = ("control", "keys", "sort", "reorder", "offsets", "density_sum", "viscous",
               "half1", "pressure", "density_relax")


class sph_domain(C.Structure):
    _fields_ = [("dim", C.c_int), ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class sph_material(C.Structure):
    _fields_ = [("rho0", C.c_double), ("c0", C.c_double), ("mu", C.c_double),
                ("U_ref", C.c_double)]


class sph_tank(C.Structure):
    _fields_ = [("domain", sph_domain), ("dp", C.c_double), ("h", C.c_double),
                ("material", sph_material), ("gravity", C.c_double * 3)]


class sph_tuning(C.Structure):
    _fields_ = [("block", C.c_int), ("radix_bits", C.c_int), ("neighbour_list", C.c_int),
                ("trials", C.c_int), ("ms_per_step", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class sph_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


class SphError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libsph.so (built in-tree by paper_2603_11868_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libsph.so not built ({p}); run __graft_entry__.build() or "
                               "python -m paper_2603_11868_gb300.build")
        L = C.CDLL(p)
        vp, i, sz, d = C.c_void_p, C.c_int, C.c_size_t, C.c_double
        L.sph_create.restype = i
        L.sph_create.argtypes = [C.POINTER(sph_domain), d, d, C.POINTER(sph_material), vp, i,
                                 C.POINTER(sph_allocator), vp, C.POINTER(vp)]
        L.sph_set_particles.restype = i
        L.sph_set_particles.argtypes = [vp, i, sz, vp, vp, vp]
        L.sph_set_wall_translation.restype = i
        L.sph_set_wall_translation.argtypes = [vp, vp]
        L.sph_set_wall_motion.restype = i
        L.sph_set_wall_motion.argtypes = [vp, vp, d, vp]
        L.sph_checkpoint_bytes.restype = sz
        L.sph_checkpoint_bytes.argtypes = [vp]
        L.sph_checkpoint_save.restype = i
        L.sph_checkpoint_save.argtypes = [vp, vp, sz]
        L.sph_checkpoint_load.restype = i
        L.sph_checkpoint_load.argtypes = [vp, vp, sz]
        L.sph_step.restype = i
        L.sph_step.argtypes = [vp, i]
        L.sph_get_fields.restype = i
        L.sph_get_fields.argtypes = [vp, C.c_uint, vp]
        L.sph_get_scalars.restype = i
        L.sph_get_scalars.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sph_count.restype = sz
        L.sph_count.argtypes = [vp, i]
        L.sph_cell_count.restype = sz
        L.sph_cell_count.argtypes = [vp]
        L.sph_debug_neighbour_state.restype = i
        L.sph_debug_neighbour_state.argtypes = [vp, vp, vp, vp, vp]
        L.sph_debug_neighbour_stats.restype = i
        L.sph_debug_neighbour_stats.argtypes = [vp, vp, vp, vp]
        L.sph_set_option.restype = i
        L.sph_set_option.argtypes = [vp, i, C.c_long]
        L.sph_synchronize.restype = i
        L.sph_synchronize.argtypes = [vp, d]
        L.sph_last_error.restype = C.c_char_p
        L.sph_last_error.argtypes = [vp]
        L.sph_destroy.restype = None
        L.sph_destroy.argtypes = [vp]
        L.sph_profile_stages.restype = i
        L.sph_profile_stages.argtypes = [vp, i, vp, vp]
        L.sph_kernels_per_step.restype = C.c_long
        L.sph_kernels_per_step.argtypes = [vp]
        L.sph_nsearch_create.restype = i
        L.sph_nsearch_create.argtypes = [C.POINTER(sph_domain), d, i, C.POINTER(sph_allocator),
                                         vp, C.POINTER(vp)]
        L.sph_nsearch_run.restype = i
        L.sph_nsearch_run.argtypes = [vp, sz, vp, vp, vp, vp]
        L.sph_nsearch_results.restype = i
        L.sph_nsearch_results.argtypes = [vp, vp, vp, vp, vp]
        L.sph_nsearch_cell_count.restype = sz
        L.sph_nsearch_cell_count.argtypes = [vp]
        L.sph_nsearch_destroy.restype = None
        L.sph_nsearch_destroy.argtypes = [vp]
        L.sph_create_batch.restype = i
        L.sph_create_batch.argtypes = [i, C.POINTER(sph_tank), i, C.POINTER(sph_allocator), vp,
                                       C.POINTER(vp)]
        L.sph_batch_set_particles.restype = i
        L.sph_batch_set_particles.argtypes = [vp, i, vp, vp, vp, vp]
        L.sph_batch_step.restype = i
        L.sph_batch_step.argtypes = [vp, i]
        L.sph_batch_get_fields.restype = i
        L.sph_batch_get_fields.argtypes = [vp, C.c_uint, vp]
        L.sph_batch_get_scalars.restype = i
        L.sph_batch_get_scalars.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sph_batch_debug_neighbour_state.restype = i
        L.sph_batch_debug_neighbour_state.argtypes = [vp, i, vp, vp, vp]
        L.sph_batch_count.restype = sz
        L.sph_batch_count.argtypes = [vp, i]
        L.sph_batch_tank_count.restype = i
        L.sph_batch_tank_count.argtypes = [vp]
        L.sph_batch_cell_count.restype = sz
        L.sph_batch_cell_count.argtypes = [vp, i]
        L.sph_batch_profile_stages.restype = i
        L.sph_batch_profile_stages.argtypes = [vp, i, vp, vp]
        L.sph_batch_kernels_per_step.restype = C.c_long
        L.sph_batch_kernels_per_step.argtypes = [vp]
        L.sph_batch_set_option.restype = i
        L.sph_batch_set_option.argtypes = [vp, i, C.c_long]
        L.sph_batch_synchronize.restype = i
        L.sph_batch_synchronize.argtypes = [vp, d]
        L.sph_batch_last_error.restype = C.c_char_p
        L.sph_batch_last_error.argtypes = [vp]
        L.sph_batch_destroy.restype = None
        L.sph_batch_destroy.argtypes = [vp]
        L.sph_debug_list_lengths.restype = i
        L.sph_debug_list_lengths.argtypes = [vp, vp]
        L.sph_autotune.restype = i
        L.sph_autotune.argtypes = [vp, i, C.POINTER(sph_tuning)]
        L.sph_batch_autotune.restype = i
        L.sph_batch_autotune.argtypes = [vp, i, C.POINTER(sph_tuning)]
        L.sph_cell_sort_noalloc.restype = i
        L.sph_cell_sort_noalloc.argtypes = [C.POINTER(sph_domain), d, vp, vp, vp, sz, vp, vp, vp,
                                            vp]
        u32 = C.c_uint32
        for name in ("sph_get_state_range", "sph_put_state_range"):
            getattr(L, name).restype = i
            getattr(L, name).argtypes = [vp, u32, sz, vp, vp, vp, vp, vp]
        L.sph_get_schedule.restype = i
        L.sph_get_schedule.argtypes = [vp, vp]
        L.sph_set_schedule.restype = i
        L.sph_set_schedule.argtypes = [vp, vp]
        L.sph_owned_vmax2.restype = i
        L.sph_owned_vmax2.argtypes = [vp, u32, C.POINTER(C.c_double)]
        L.sph_set_vmax2.restype = i
        L.sph_set_vmax2.argtypes = [vp, d]
        for name in ("sph_get_state_rows_device", "sph_put_state_rows_device"):
            getattr(L, name).restype = i
            getattr(L, name).argtypes = [vp, u32, sz, vp]
        L.sph_owned_vmax2_device.restype = i
        L.sph_owned_vmax2_device.argtypes = [vp, u32, vp]
        L.sph_set_vmax2_device.restype = i
        L.sph_set_vmax2_device.argtypes = [vp, vp]
        _lib = L
        return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(ctx, rc):
    if rc != SPH_OK:
        msg = load().sph_last_error(ctx).decode() if ctx else ""
        raise SphError(rc, msg)


def _check_batch(b, rc):
    if rc != SPH_OK:
        msg = load().sph_batch_last_error(b).decode() if b else ""
        raise SphError(rc, msg)


# --- the C entry points, same names --------------------------------------
def sph_create(dim, lo, hi, dp, h, rho0, c0, mu, U_ref, gravity, precision=SPH_MIXED,
               allocator: sph_allocator | None = None, stream: int = 0):
    L = load()
    dom = sph_domain(int(dim), (C.c_double * 3)(*list(lo) + [0.0] * (3 - len(lo))),
                     (C.c_double * 3)(*list(hi) + [0.0] * (3 - len(hi))))
    mat = sph_material(rho0, c0, mu, U_ref)
    g = np.zeros(3)
    g[: len(gravity)] = gravity
    out = C.c_void_p()
    rc = L.sph_create(C.byref(dom), dp, h, C.byref(mat), _ptr(g), int(precision),
                      C.byref(allocator) if allocator is not None else None,
                      C.c_void_p(stream) if stream else None, C.byref(out))
    _check(None, rc)
    return out.value


def sph_set_particles(ctx, kind, pos, vel=None, rho=None):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
    rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    _check(ctx, load().sph_set_particles(ctx, int(kind), len(pos), _ptr(pos), _ptr(vel),
                                         _ptr(rho)))


def sph_set_wall_translation(ctx, moves=None):
    moves = None if moves is None else np.ascontiguousarray(moves, dtype=np.uint8)
    _check(ctx, load().sph_set_wall_translation(ctx, _ptr(moves)))


def sph_set_wall_motion(ctx, moves, omega=0.0, amplitude=None):
    moves = None if moves is None else np.ascontiguousarray(moves, dtype=np.uint8)
    amplitude = None if amplitude is None else np.ascontiguousarray(amplitude,
                                                                     dtype=np.float64)
    _check(ctx, load().sph_set_wall_motion(ctx, _ptr(moves), float(omega), _ptr(amplitude)))


def sph_checkpoint_save(ctx):
    n = load().sph_checkpoint_bytes(ctx)
    buf = np.empty(n, dtype=np.uint8)
    _check(ctx, load().sph_checkpoint_save(ctx, _ptr(buf), n))
    return buf


def sph_checkpoint_load(ctx, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(ctx, load().sph_checkpoint_load(ctx, _ptr(buf), buf.size))


def sph_step(ctx, n):
    _check(ctx, load().sph_step(ctx, int(n)))


def sph_get_fields(ctx, mask, n, dim):
    comps = sum(dim if (mask & b) and b in _VECTOR_FIELDS else (1 if mask & b else 0)
                for b in (1 << k for k in range(8)))
    out = np.empty(n * comps, dtype=np.float64)
    _check(ctx, load().sph_get_fields(ctx, int(mask), _ptr(out)))
    res, off = {}, 0
    for name, b in FIELD_NAMES.items():
        if mask & b:
            c = dim if b in _VECTOR_FIELDS else 1
            a = out[off: off + n * c]
            res[name] = a.reshape(n, dim) if c > 1 else a
            off += n * c
    return res


def sph_get_scalars(ctx):
    t, dta, dtc = C.c_double(), C.c_double(), C.c_double()
    nac, nad = C.c_long(), C.c_long()
    _check(ctx, load().sph_get_scalars(ctx, C.byref(t), C.byref(dta), C.byref(dtc),
                                       C.byref(nac), C.byref(nad)))
    return dict(t=t.value, dt_ad=dta.value, dt_ac=dtc.value, n_ac=nac.value, n_adv=nad.value)


def sph_count(ctx, kind=SPH_FLUID):
    return load().sph_count(ctx, int(kind))


def sph_cell_count(ctx):
    return load().sph_cell_count(ctx)


def sph_debug_neighbour_state(ctx, n, ncell):
    keys = np.empty(n, np.uint32); perm = np.empty(n, np.uint32)
    ids = np.empty(n, np.uint32); cb = np.empty(ncell + 1, np.uint32)
    _check(ctx, load().sph_debug_neighbour_state(ctx, _ptr(keys), _ptr(perm), _ptr(ids),
                                                 _ptr(cb)))
    return dict(keys=keys, perm=perm, ids=ids, cell_begin=cb)


def sph_debug_neighbour_stats(ctx, n):
    cf = np.empty(n, np.uint32); cw = np.empty(n, np.uint32); hs = np.empty(n, np.uint64)
    _check(ctx, load().sph_debug_neighbour_stats(ctx, _ptr(cf), _ptr(cw), _ptr(hs)))
    return cf, cw, hs


STATE_FIELDS = ("pos", "vel", "rho", "drho", "aprior")


def sph_get_state_range(ctx, id0, m, dim):
    """State of user ids [id0, id0 + m): dict of pos, vel (m, dim), rho, drho (m),
    aprior (m, dim), float64."""
    out = {"pos": np.empty((m, dim)), "vel": np.empty((m, dim)), "rho": np.empty(m),
           "drho": np.empty(m), "aprior": np.empty((m, dim))}
    _check(ctx, load().sph_get_state_range(ctx, id0, m, *(_ptr(out[k]) for k in STATE_FIELDS)))
    return out


def sph_put_state_range(ctx, id0, state):
    """Write the state of user ids [id0, id0 + m) (dict as sph_get_state_range
    returns; missing keys are left as they are)."""
    arr = {k: (np.ascontiguousarray(state[k], dtype=np.float64) if state.get(k) is not None
               else None) for k in STATE_FIELDS}
    m = len(next(a for a in arr.values() if a is not None)) if any(
        a is not None for a in arr.values()) else 0
    _check(ctx, load().sph_put_state_range(ctx, id0, m, *(_ptr(arr[k]) for k in STATE_FIELDS)))


SCHEDULE_KEYS = ("t", "tau", "dt_ad", "dt_ac", "n_ac", "n_adv", "started", "vmax2")


def sph_get_schedule(ctx):
    out = np.zeros(8)
    _check(ctx, load().sph_get_schedule(ctx, _ptr(out)))
    return dict(zip(SCHEDULE_KEYS, out.tolist()))


def sph_set_schedule(ctx, sched):
    arr = np.array([float(sched[k]) for k in SCHEDULE_KEYS])
    _check(ctx, load().sph_set_schedule(ctx, _ptr(arr)))


def sph_owned_vmax2(ctx, n_own):
    v = C.c_double()
    _check(ctx, load().sph_owned_vmax2(ctx, int(n_own), C.byref(v)))
    return v.value


def sph_set_vmax2(ctx, vmax2):
    _check(ctx, load().sph_set_vmax2(ctx, float(vmax2)))


def sph_debug_list_lengths(ctx, n):
    out = np.empty(n, np.uint32)
    _check(ctx, load().sph_debug_list_lengths(ctx, _ptr(out)))
    return out


def sph_set_option(ctx, option, value):
    _check(ctx, load().sph_set_option(ctx, int(option), int(value)))


def sph_synchronize(ctx, timeout_s=0.0):
    _check(ctx, load().sph_synchronize(ctx, float(timeout_s)))


def sph_last_error(ctx):
    return load().sph_last_error(ctx).decode()


def sph_destroy(ctx):
    load().sph_destroy(ctx)


def sph_profile_stages(ctx, n):
    ms = np.zeros(len(STAGE_NAMES), np.float64)
    reb = C.c_long()
    _check(ctx, load().sph_profile_stages(ctx, int(n), _ptr(ms), C.byref(reb)))
    return dict(zip(STAGE_NAMES, ms)), reb.value


def sph_kernels_per_step(ctx):
    return load().sph_kernels_per_step(ctx)


def sph_autotune(ctx, steps_per_trial=10):
    t = sph_tuning()
    _check(ctx, load().sph_autotune(ctx, int(steps_per_trial), C.byref(t)))
    return t.as_dict()


class TuningCache:
    """Autotuner choices kept in a JSON file, keyed by the GPU's name and the
    problem's configuration (dimension, precision, particle and wall counts,
    cell grid, smoothing length), so that a later run of the same problem on
    the same kind of GPU takes the choice without the trials."""

    def __init__(self, path: str):
        self.path = path

    @staticmethod
    def key(obj) -> str:
        import torch
        gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
        cfg = obj.tuning_signature()
        return gpu + "|" + ",".join(f"{k}={cfg[k]}" for k in sorted(cfg))

    def _read(self) -> dict:
        import json
        try:
            with open(self.path) as fh:
                return json.load(fh)
        except (OSError, ValueError):
            return {}

    def get(self, obj):
        return self._read().get(self.key(obj))

    def put(self, obj, tuning: dict) -> None:
        import json
        data = self._read()
        data[self.key(obj)] = {k: int(tuning[k]) for k in ("block", "radix_bits",
                                                           "neighbour_list")}
        tmp = self.path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def tune(obj, steps_per_trial=10, cache: str | None = None) -> dict:
    """Autotune a Solver or Batch, or take a cached choice (TuningCache)."""
    if cache:
        tc = TuningCache(cache)
        hit = tc.get(obj)
        if hit:
            obj.set_option(SPH_OPT_BLOCK, hit["block"])
            obj.set_option(SPH_OPT_RADIX_BITS, hit["radix_bits"])
            obj.set_option(SPH_OPT_NEIGHBOUR_LIST, hit["neighbour_list"])
            return dict(hit, trials=0, cached=True)
    t = obj.autotune(steps_per_trial)
    if cache:
        TuningCache(cache).put(obj, t)
    return t


class NeighbourSearch:
    """sph_nsearch_*: keys, radix sort, reorder, offsets and one density pass
    over device positions (torch tensors, float32 or float64)."""

    STAGES = ("keys", "sort", "reorder", "offsets", "density")

    def __init__(self, dim, lo, hi, h, fp32=False, torch_memory=True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the SPH library has no CPU path")
        L = load()
        self._allocator = TorchAllocator() if torch_memory else None
        dom = sph_domain(int(dim), (C.c_double * 3)(*list(lo) + [0.0] * (3 - len(lo))),
                         (C.c_double * 3)(*list(hi) + [0.0] * (3 - len(hi))))
        out = C.c_void_p()
        rc = L.sph_nsearch_create(C.byref(dom), float(h), SPH_MIXED if fp32 else SPH_FP64,
                                  C.byref(self._allocator.struct) if self._allocator else None,
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream) or None,
                                  C.byref(out))
        _check(None, rc)
        self.ns = out.value
        self.dim = int(dim)
        self.n = 0

    @property
    def ncell(self):
        return load().sph_nsearch_cell_count(self.ns)

    def run(self, x, y, z=None, timed=True):
        """x, y, z: contiguous device tensors of one dtype; returns the stage
        times in ms (when timed)."""
        ms = np.zeros(5, np.float64) if timed else None
        self.n = int(x.numel())
        zp = z.data_ptr() if z is not None else None
        _check(None, load().sph_nsearch_run(self.ns, self.n, x.data_ptr(), y.data_ptr(), zp,
                                             _ptr(ms)))
        return dict(zip(self.STAGES, ms)) if timed else None

    def results(self):
        n = self.n
        keys = np.empty(n, np.uint32); perm = np.empty(n, np.uint32)
        cb = np.empty(self.ncell + 1, np.uint32); sig = np.empty(n, np.float64)
        _check(None, load().sph_nsearch_results(self.ns, _ptr(keys), _ptr(perm), _ptr(cb),
                                                 _ptr(sig)))
        return dict(keys=keys, perm=perm, cell_begin=cb, sigma=sig)

    def close(self):
        if getattr(self, "ns", None):
            load().sph_nsearch_destroy(self.ns)
            self.ns = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- batches of independent tanks -----------------------------------------
def _domain_of(dim, lo, hi):
    return sph_domain(int(dim), (C.c_double * 3)(*list(lo) + [0.0] * (3 - len(lo))),
                      (C.c_double * 3)(*list(hi) + [0.0] * (3 - len(hi))))


def sph_create_batch(cases, precision=SPH_MIXED, allocator: sph_allocator | None = None,
                     stream: int = 0):
    """cases: sequence of objects with the attributes of ``cases.Case``."""
    tanks = (sph_tank * len(cases))()
    for t, c in enumerate(cases):
        g = list(c.gravity) + [0.0] * (3 - len(c.gravity))
        tanks[t] = sph_tank(_domain_of(c.dim, c.lo, c.hi), float(c.dp), float(c.h),
                            sph_material(c.rho0, c.c0, c.mu, c.U_ref), (C.c_double * 3)(*g))
    out = C.c_void_p()
    rc = load().sph_create_batch(len(cases), tanks, int(precision),
                                 C.byref(allocator) if allocator is not None else None,
                                 C.c_void_p(stream) if stream else None, C.byref(out))
    _check_batch(None, rc)
    return out.value


def sph_batch_set_particles(b, kind, counts, pos, vel=None, rho=None):
    counts = np.ascontiguousarray(counts, dtype=np.uint64)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
    rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
    _check_batch(b, load().sph_batch_set_particles(b, int(kind), _ptr(counts), _ptr(pos),
                                                   _ptr(vel), _ptr(rho)))


def sph_batch_step(b, n):
    _check_batch(b, load().sph_batch_step(b, int(n)))


def sph_batch_get_fields(b, mask, n, dim):
    comps = sum(dim if (mask & f) and f in _VECTOR_FIELDS else (1 if mask & f else 0)
                for f in (1 << k for k in range(8)))
    out = np.empty(n * comps, dtype=np.float64)
    _check_batch(b, load().sph_batch_get_fields(b, int(mask), _ptr(out)))
    res, off = {}, 0
    for name, f in FIELD_NAMES.items():
        if mask & f:
            c = dim if f in _VECTOR_FIELDS else 1
            a = out[off: off + n * c]
            res[name] = a.reshape(n, dim) if c > 1 else a
            off += n * c
    return res


def sph_batch_get_scalars(b, n_tanks):
    t, dta, dtc = (np.empty(n_tanks, np.float64) for _ in range(3))
    nac, nad = np.empty(n_tanks, np.int64), np.empty(n_tanks, np.int64)
    _check_batch(b, load().sph_batch_get_scalars(b, _ptr(t), _ptr(dta), _ptr(dtc), _ptr(nac),
                                                 _ptr(nad)))
    return dict(t=t, dt_ad=dta, dt_ac=dtc, n_ac=nac, n_adv=nad)


def sph_batch_debug_neighbour_state(b, tank, n, ncell):
    keys = np.empty(n, np.uint32); ids = np.empty(n, np.uint32)
    cb = np.empty(ncell + 1, np.uint32)
    _check_batch(b, load().sph_batch_debug_neighbour_state(b, int(tank), _ptr(keys), _ptr(ids),
                                                           _ptr(cb)))
    return dict(keys=keys, ids=ids, cell_begin=cb)


def sph_batch_count(b, kind=SPH_FLUID):
    return load().sph_batch_count(b, int(kind))


def sph_batch_tank_count(b):
    return load().sph_batch_tank_count(b)


def sph_batch_cell_count(b, tank):
    return load().sph_batch_cell_count(b, int(tank))


def sph_batch_profile_stages(b, n):
    ms = np.zeros(len(STAGE_NAMES), np.float64)
    reb = C.c_long()
    _check_batch(b, load().sph_batch_profile_stages(b, int(n), _ptr(ms), C.byref(reb)))
    return dict(zip(STAGE_NAMES, ms)), reb.value


def sph_batch_kernels_per_step(b):
    return load().sph_batch_kernels_per_step(b)


def sph_batch_set_option(b, option, value):
    _check_batch(b, load().sph_batch_set_option(b, int(option), int(value)))


def sph_batch_synchronize(b, timeout_s=0.0):
    _check_batch(b, load().sph_batch_synchronize(b, float(timeout_s)))


def sph_batch_last_error(b):
    return load().sph_batch_last_error(b).decode()


def sph_batch_destroy(b):
    load().sph_batch_destroy(b)


def sph_batch_autotune(b, steps_per_trial=10):
    t = sph_tuning()
    _check_batch(b, load().sph_batch_autotune(b, int(steps_per_trial), C.byref(t)))
    return t.as_dict()


class Batch:
    """A batch of independent tanks (``cases``: a list of ``cases.Case``), each
    with its own particles and schedule.  Fields come back tank-major."""

    def __init__(self, cases, precision: str = "mixed", torch_memory: bool = True,
                 stream: int | None = None):
        self.cases = list(cases)
        if any(getattr(c, "wall_moves", None) is not None and np.any(c.wall_moves)
               for c in self.cases):
            raise ValueError("batches have no translating walls (sph_set_wall_translation "
                             "is a single-tank call)")
        self.dim = self.cases[0].dim
        self.precision = SPH_FP64 if precision == "fp64" else SPH_MIXED
        self._allocator = None
        if torch_memory:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device: the SPH library has no CPU path")
            self._allocator = TorchAllocator()
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
        self.b = sph_create_batch(self.cases, self.precision,
                                  self._allocator.struct if self._allocator else None,
                                  stream or 0)
        self.counts = np.array([c.n for c in self.cases], dtype=np.int64)
        self.offsets = np.concatenate([[0], np.cumsum(self.counts)])
        walls = [c.wall if c.wall is not None else np.zeros((0, self.dim)) for c in self.cases]
        wcounts = [len(w) for w in walls]
        if sum(wcounts):
            wvel = None if all(getattr(c, "wall_vel", None) is None for c in self.cases) else \
                np.concatenate([c.wall_vel if getattr(c, "wall_vel", None) is not None
                                else np.zeros_like(w) for c, w in zip(self.cases, walls)])
            sph_batch_set_particles(self.b, SPH_WALL, wcounts, np.concatenate(walls), wvel)
        vel = None if all(c.vel is None for c in self.cases) else np.concatenate(
            [c.vel if c.vel is not None else np.zeros_like(c.fluid) for c in self.cases])
        rho = None if all(c.rho is None for c in self.cases) else np.concatenate(
            [c.rho if c.rho is not None else np.full(c.n, c.rho0) for c in self.cases])
        sph_batch_set_particles(self.b, SPH_FLUID, self.counts,
                                np.concatenate([c.fluid for c in self.cases]), vel, rho)

    @property
    def tanks(self):
        return len(self.cases)

    @property
    def n(self):
        return sph_batch_count(self.b, SPH_FLUID)

    @property
    def nw(self):
        return sph_batch_count(self.b, SPH_WALL)

    def step(self, n: int = 1):
        sph_batch_step(self.b, n)

    def fields(self, *names):
        mask = 0
        for nm in names:
            mask |= FIELD_NAMES[nm]
        return sph_batch_get_fields(self.b, mask, self.n, self.dim)

    def tank_fields(self, tank, *names):
        f = self.fields(*names)
        a, e = self.offsets[tank], self.offsets[tank + 1]
        return {k: v[a:e] for k, v in f.items()}

    def scalars(self):
        return sph_batch_get_scalars(self.b, self.tanks)

    def set_option(self, option, value):
        sph_batch_set_option(self.b, option, value)

    def neighbour_state(self, tank):
        n = int(self.counts[tank]) if 0 <= tank < self.tanks else 0
        return sph_batch_debug_neighbour_state(self.b, tank, n,
                                               sph_batch_cell_count(self.b, tank))

    def profile(self, n):
        return sph_batch_profile_stages(self.b, n)

    def autotune(self, steps_per_trial=10):
        return sph_batch_autotune(self.b, steps_per_trial)

    def synchronize(self, timeout_s=0.0):
        sph_batch_synchronize(self.b, timeout_s)

    def tuning_signature(self) -> dict:
        return {"kind": "batch", "dim": self.dim, "precision": int(self.precision),
                "tanks": self.tanks, "n": self.n, "nw": self.nw}

    def close(self):
        if getattr(self, "b", None):
            sph_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sph_cell_sort_noalloc(dim, lo, hi, cell_size, x, y, z, n, keys_out, perm_out,
                          cell_begin_out, stream=0):
    """Device-pointer arguments (ints); returns the status code (no raise)."""
    dom = sph_domain(int(dim), (C.c_double * 3)(*list(lo) + [0.0] * (3 - len(lo))),
                     (C.c_double * 3)(*list(hi) + [0.0] * (3 - len(hi))))
    return load().sph_cell_sort_noalloc(C.byref(dom), float(cell_size), x, y, z, int(n),
                                        keys_out, perm_out, cell_begin_out,
                                        C.c_void_p(stream) if stream else None)


# --- PyTorch plumbing ------------------------------------------------------
class TorchAllocator:
    """Allocator callbacks backed by torch's CUDA caching allocator."""

    def __init__(self, device: int | None = None):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else int(device)
        self._alloc = ALLOC_FN(self._on_alloc)
        self._free = FREE_FN(self._on_free)
        self.struct = sph_allocator(self._alloc, self._free, None)

    def _on_alloc(self, nbytes, stream, user):
        try:
            return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                            stream=int(stream or 0))
        except Exception:  # out of memory -> NULL -> SPH_E_OOM
            return None

    def _on_free(self, ptr, nbytes, stream, user):
        self._torch.cuda.caching_allocator_delete(int(ptr))


class Solver:
    """One SPH context.  ``case`` is a ``cases.Case`` (or anything with the same
    attributes).  ``precision`` is "fp64" or "mixed"."""

    def __init__(self, case, precision: str = "mixed", torch_memory: bool = True,
                 stream: int | None = None):
        self.case = case
        self.dim = case.dim
        self.precision = SPH_FP64 if precision == "fp64" else SPH_MIXED
        self._allocator = None
        if torch_memory:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device: the SPH library has no CPU path")
            self._allocator = TorchAllocator()
            if stream is None:
                stream = torch.cuda.current_stream().cuda_stream
        self.ctx = sph_create(case.dim, case.lo, case.hi, case.dp, case.h, case.rho0, case.c0,
                              case.mu, case.U_ref, case.gravity, self.precision,
                              self._allocator.struct if self._allocator else None, stream or 0)
        if case.wall is not None and len(case.wall):
            sph_set_particles(self.ctx, SPH_WALL, case.wall, getattr(case, "wall_vel", None))
            if getattr(case, "wall_moves", None) is not None:
                sph_set_wall_motion(self.ctx, case.wall_moves, getattr(case, "wall_omega", 0.0),
                                    getattr(case, "wall_amplitude", None))
        sph_set_particles(self.ctx, SPH_FLUID, case.fluid, case.vel, case.rho)

    @property
    def n(self):
        return sph_count(self.ctx, SPH_FLUID)

    @property
    def nw(self):
        return sph_count(self.ctx, SPH_WALL)

    @property
    def ncell(self):
        return sph_cell_count(self.ctx)

    def set_fluid(self, pos, vel=None, rho=None):
        sph_set_particles(self.ctx, SPH_FLUID, pos, vel, rho)

    def step(self, n: int = 1):
        sph_step(self.ctx, n)

    def fields(self, *names):
        mask = 0
        for nm in names:
            mask |= FIELD_NAMES[nm]
        return sph_get_fields(self.ctx, mask, self.n, self.dim)

    def field(self, name):
        return self.fields(name)[name]

    def scalars(self):
        return sph_get_scalars(self.ctx)

    def set_option(self, option, value):
        sph_set_option(self.ctx, option, value)

    def neighbour_state(self):
        return sph_debug_neighbour_state(self.ctx, self.n, self.ncell)

    def autotune(self, steps_per_trial=10):
        return sph_autotune(self.ctx, steps_per_trial)

    def list_lengths(self):
        return sph_debug_list_lengths(self.ctx, self.n)

    def neighbour_stats(self):
        return sph_debug_neighbour_stats(self.ctx, self.n)

    def tuning_signature(self) -> dict:
        c = self.case
        return {"kind": "tank", "dim": c.dim, "precision": int(self.precision), "n": self.n,
                "nw": self.nw, "cells": self.ncell, "h_over_dp": round(c.h / c.dp, 6)}

    def checkpoint(self) -> np.ndarray:
        """The run's state as a byte array (sph_checkpoint_save)."""
        return sph_checkpoint_save(self.ctx)

    def restore(self, buf) -> None:
        """Continue from a checkpoint of a solver with the same setup."""
        sph_checkpoint_load(self.ctx, buf)

    def profile_stages(self, n: int):
        return sph_profile_stages(self.ctx, n)

    def kernels_per_step(self):
        return sph_kernels_per_step(self.ctx)

    def synchronize(self, timeout_s=0.0):
        sph_synchronize(self.ctx, timeout_s)

    def close(self):
        if getattr(self, "ctx", None):
            sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
