"""ctypes loader for the serial FP64 oracle (oracle/sph_oracle.c).

TEST INFRASTRUCTURE ONLY.  Imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the product package.
It shares no code with the CUDA library: it compiles and calls the plain C
restatement of the method in this folder.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_HDR = os.path.join(_HERE, "sph_oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

# field ids, mirror of the enum in sph_oracle.h
POS, VEL, RHO, P, DRHO, ACC, APRIOR, SIGMA = range(8)
_VECTOR = {POS, VEL, ACC, APRIOR}


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (-ffp-contract=off: no fused multiply-add,
    so x86 and Arm hosts produce the same bits)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    stale = (not os.path.exists(_OUT) or
             os.path.getmtime(_OUT) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
    if force or stale:
        tmp = _OUT + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # a test may point the loader at a deliberately mutated build
            path = os.environ.get("ORACLE_LIB_OVERRIDE") or build()
            L = C.CDLL(path)
            d, i, l, vp = C.c_double, C.c_int, C.c_long, C.c_void_p
            dp = C.POINTER(C.c_double)
            L.osph_alpha.restype = d; L.osph_alpha.argtypes = [i, d]
            L.osph_W.restype = d; L.osph_W.argtypes = [i, d, d]
            L.osph_dW.restype = d; L.osph_dW.argtypes = [i, d, d]
            L.osph_sigma0.restype = d; L.osph_sigma0.argtypes = [i, d, d]
            L.osph_riemann.restype = None
            L.osph_riemann.argtypes = [d, d, d, d, d, d, d, dp, dp]
            L.osph_create.restype = vp
            L.osph_create.argtypes = [i, vp, vp, d, d, d, d, d, d, vp]
            L.osph_destroy.restype = None; L.osph_destroy.argtypes = [vp]
            L.osph_set_particles.restype = i
            L.osph_set_particles.argtypes = [vp, i, l, vp, vp, vp]
            L.osph_set_drho.restype = i; L.osph_set_drho.argtypes = [vp, vp]
            L.osph_set_wall_translation.restype = i
            L.osph_set_wall_translation.argtypes = [vp, vp]
            L.osph_set_wall_motion.restype = i
            L.osph_set_wall_motion.argtypes = [vp, vp, d, vp]
            L.osph_set_time.restype = None
            L.osph_set_time.argtypes = [vp, d]
            L.osph_set_variant.restype = None; L.osph_set_variant.argtypes = [vp, i, i]
            L.osph_set_transport_correction.restype = None
            L.osph_set_transport_correction.argtypes = [vp, i]
            L.osph_transport_correction.restype = None
            L.osph_transport_correction.argtypes = [vp]
            L.osph_step.restype = i; L.osph_step.argtypes = [vp, l]
            for name in ("osph_rebuild", "osph_density_summation", "osph_viscous"):
                getattr(L, name).restype = None
                getattr(L, name).argtypes = [vp]
            L.osph_vmax2.restype = d; L.osph_vmax2.argtypes = [vp]
            for name in ("osph_half1", "osph_pressure_relaxation", "osph_half2"):
                getattr(L, name).restype = None
                getattr(L, name).argtypes = [vp, d]
            L.osph_get_field.restype = i; L.osph_get_field.argtypes = [vp, i, vp]
            L.osph_get_scalars.restype = None
            L.osph_get_scalars.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
            for name in ("osph_n", "osph_nw", "osph_ncell"):
                getattr(L, name).restype = l
                getattr(L, name).argtypes = [vp]
            L.osph_grid.restype = None; L.osph_grid.argtypes = [vp, vp, vp]
            L.osph_neighbour_state.restype = None
            L.osph_neighbour_state.argtypes = [vp, vp, vp, vp, vp]
            L.osph_wall_state.restype = None
            L.osph_wall_state.argtypes = [vp, vp, vp, vp]
            L.osph_neighbour_stats.restype = None
            L.osph_neighbour_stats.argtypes = [vp, i, vp, vp, vp]
            L.osph_front_ke.restype = None; L.osph_front_ke.argtypes = [vp, vp, vp]
            L.osph_sample_sigma.restype = None
            L.osph_sample_sigma.argtypes = [vp, l, vp, vp]
            L.osph_sample_first_step_acc.restype = None
            L.osph_sample_first_step_acc.argtypes = [vp, l, vp, vp]
            L.osph_state_range.restype = i
            L.osph_state_range.argtypes = [vp, l, l, vp, vp, vp, vp, vp, i]
            L.osph_set_schedule.restype = None
            L.osph_set_schedule.argtypes = [vp, d, d, d, d, l, l, i]
            _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _vec3(v) -> np.ndarray:
    out = np.zeros(3, dtype=np.float64)
    out[: len(v)] = v
    return out


def W(dim: int, h: float, r: float) -> float:
    return lib().osph_W(dim, h, r)


def dW(dim: int, h: float, r: float) -> float:
    return lib().osph_dW(dim, h, r)


def alpha(dim: int, h: float) -> float:
    return lib().osph_alpha(dim, h)


def sigma0(dim: int, dp: float, h: float) -> float:
    return lib().osph_sigma0(dim, dp, h)


def riemann(pL, pR, rhoL, rhoR, UL, UR, c0):
    Ps, Us = C.c_double(), C.c_double()
    lib().osph_riemann(pL, pR, rhoL, rhoR, UL, UR, c0, C.byref(Ps), C.byref(Us))
    return Ps.value, Us.value


class Oracle:
    """One simulation held by the C oracle.  Arrays in and out are in user
    order (the order given to ``set_fluid``)."""

    def __init__(self, dim, lo, hi, dp, h, rho0, c0, mu, U_ref, gravity):
        self.dim = int(dim)
        self._lo, self._hi, self._g = _vec3(lo), _vec3(hi), _vec3(gravity)
        self.dp, self.h, self.rho0, self.c0, self.mu = dp, h, rho0, c0, mu
        self._s = lib().osph_create(self.dim, _ptr(self._lo), _ptr(self._hi), dp, h, rho0,
                                    c0, mu, U_ref, _ptr(self._g))
        if not self._s:
            raise ValueError("oracle: bad arguments")

    @classmethod
    def from_case(cls, case, set_particles: bool = True):
        o = cls(case.dim, case.lo, case.hi, case.dp, case.h, case.rho0, case.c0, case.mu,
                case.U_ref, case.gravity)
        if set_particles:
            if case.wall is not None and len(case.wall):
                o.set_wall(case.wall, case.wall_vel)
                if getattr(case, "wall_moves", None) is not None:
                    o.set_wall_motion(case.wall_moves, getattr(case, "wall_omega", 0.0),
                                      getattr(case, "wall_amplitude", None))
            o.set_fluid(case.fluid, case.vel, case.rho)
        return o

    def __del__(self):
        s = getattr(self, "_s", None)
        if s:
            lib().osph_destroy(s)
            self._s = None

    def set_fluid(self, pos, vel=None, rho=None):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        vel = None if vel is None else np.ascontiguousarray(vel, dtype=np.float64)
        rho = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64)
        rc = lib().osph_set_particles(self._s, 0, len(pos), _ptr(pos), _ptr(vel), _ptr(rho))
        if rc:
            raise ValueError("oracle: set_particles failed")

    def set_wall(self, pos, vel=None):
        """Wall particles; vel = prescribed velocity of a sliding wall (None = rest)."""
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        if vel is not None:
            vel = np.ascontiguousarray(vel, dtype=np.float64)
            assert vel.shape == pos.shape
        if lib().osph_set_particles(self._s, 1, len(pos), _ptr(pos), _ptr(vel), None):
            raise ValueError("oracle: set_particles (wall) failed")

    def set_wall_translation(self, moves):
        """moves[u] != 0: wall u moves with its velocity (None clears)."""
        if moves is not None:
            moves = np.ascontiguousarray(moves, dtype=np.uint8)
        lib().osph_set_wall_translation(self._s, _ptr(moves))

    def set_wall_motion(self, moves, omega=0.0, amplitude=None):
        """Translating walls (moves[u] != 0) that also oscillate with
        amplitude[u] at angular frequency omega (None: uniform motion)."""
        if moves is not None:
            moves = np.ascontiguousarray(moves, dtype=np.uint8)
        if amplitude is not None:
            amplitude = np.ascontiguousarray(amplitude, dtype=np.float64)
        lib().osph_set_wall_motion(self._s, _ptr(moves), float(omega), _ptr(amplitude))

    def set_time(self, t):
        """Sets the simulation time (translating walls placed at it)."""
        lib().osph_set_time(self._s, float(t))

    def set_drho(self, drho):
        drho = np.ascontiguousarray(drho, dtype=np.float64)
        lib().osph_set_drho(self._s, _ptr(drho))

    def set_transport_correction(self, on: bool = True):
        """Transport-velocity correction once per advection step."""
        lib().osph_set_transport_correction(self._s, int(bool(on)))

    def transport_correction(self):
        lib().osph_transport_correction(self._s)

    def set_variant(self, density_riemann: bool = True, reinit_blended: bool = False):
        """Method variants: Riemann or averaged U* in the density relaxation;
        clamped or blended free-surface density reinitialisation."""
        lib().osph_set_variant(self._s, int(bool(density_riemann)), int(bool(reinit_blended)))

    @property
    def n(self):
        return lib().osph_n(self._s)

    @property
    def nw(self):
        return lib().osph_nw(self._s)

    @property
    def ncell(self):
        return lib().osph_ncell(self._s)

    def grid(self):
        cs = C.c_double()
        nc = np.zeros(3, dtype=np.int64)
        lib().osph_grid(self._s, C.byref(cs), _ptr(nc))
        return cs.value, nc

    def step(self, n: int = 1) -> int:
        return lib().osph_step(self._s, int(n))

    # stages
    def rebuild(self):
        lib().osph_rebuild(self._s)

    def density_summation(self):
        lib().osph_density_summation(self._s)

    def viscous(self):
        lib().osph_viscous(self._s)

    def vmax2(self):
        return lib().osph_vmax2(self._s)

    def half1(self, dt):
        lib().osph_half1(self._s, dt)

    def pressure_relaxation(self, dt):
        lib().osph_pressure_relaxation(self._s, dt)

    def half2(self, dt):
        lib().osph_half2(self._s, dt)

    def field(self, fid: int) -> np.ndarray:
        shape = (self.n, self.dim) if fid in _VECTOR else (self.n,)
        out = np.zeros(shape, dtype=np.float64)
        if lib().osph_get_field(self._s, fid, _ptr(out)) < 0:
            raise ValueError(f"oracle: unknown field {fid}")
        return out

    def scalars(self) -> dict:
        t, tau, dta, dtc = (C.c_double() for _ in range(4))
        nac, nad = C.c_long(), C.c_long()
        fl = C.c_int()
        lib().osph_get_scalars(self._s, C.byref(t), C.byref(tau), C.byref(dta), C.byref(dtc),
                               C.byref(nac), C.byref(nad), C.byref(fl))
        return dict(t=t.value, tau=tau.value, dt_ad=dta.value, dt_ac=dtc.value,
                    n_ac=nac.value, n_adv=nad.value, flags=fl.value)

    def neighbour_state(self):
        n, nc = self.n, self.ncell
        keys = np.zeros(n, np.uint32); perm = np.zeros(n, np.uint32)
        ids = np.zeros(n, np.uint32); cb = np.zeros(nc + 1, np.uint32)
        lib().osph_neighbour_state(self._s, _ptr(keys), _ptr(perm), _ptr(ids), _ptr(cb))
        return dict(keys=keys, perm=perm, ids=ids, cell_begin=cb)

    def wall_state(self):
        nw, nc = self.nw, self.ncell
        keys = np.zeros(nw, np.uint32); ids = np.zeros(nw, np.uint32)
        cb = np.zeros(nc + 1, np.uint32)
        lib().osph_wall_state(self._s, _ptr(keys), _ptr(ids), _ptr(cb))
        return dict(keys=keys, ids=ids, cell_begin=cb)

    def neighbour_stats(self, brute: bool = False):
        n = self.n
        cf = np.zeros(n, np.uint32); cw = np.zeros(n, np.uint32); hs = np.zeros(n, np.uint64)
        lib().osph_neighbour_stats(self._s, int(brute), _ptr(cf), _ptr(cw), _ptr(hs))
        return cf, cw, hs

    def front_ke(self):
        f, k = C.c_double(), C.c_double()
        lib().osph_front_ke(self._s, C.byref(f), C.byref(k))
        return f.value, k.value

    def sample_first_step_acc(self, user_ids):
        ids = np.ascontiguousarray(user_ids, dtype=np.uint32)
        out = np.zeros((len(ids), self.dim), np.float64)
        lib().osph_sample_first_step_acc(self._s, len(ids), _ptr(ids), _ptr(out))
        return out

    def state_range(self, id0, m):
        """State of user ids [id0, id0 + m): pos, vel, aprior (m, dim), rho, drho (m)."""
        out = {k: np.zeros((m, 3)) for k in ("pos", "vel", "aprior")}
        out.update(rho=np.zeros(m), drho=np.zeros(m))
        if lib().osph_state_range(self._s, id0, m, _ptr(out["pos"]), _ptr(out["vel"]),
                                  _ptr(out["rho"]), _ptr(out["drho"]), _ptr(out["aprior"]), 0):
            raise ValueError("oracle: id range beyond n")
        for k in ("pos", "vel", "aprior"):
            out[k] = np.ascontiguousarray(out[k][:, :self.dim])
        return out

    def put_state_range(self, id0, state):
        """Write the state of user ids [id0, id0 + m) (keys as state_range)."""
        m = len(state["rho"])
        full = {}
        for k in ("pos", "vel", "aprior"):
            a = np.zeros((m, 3))
            a[:, :self.dim] = state[k]
            full[k] = a
        rho = np.ascontiguousarray(state["rho"], dtype=np.float64)
        drho = np.ascontiguousarray(state["drho"], dtype=np.float64)
        if lib().osph_state_range(self._s, id0, m, _ptr(full["pos"]), _ptr(full["vel"]),
                                  _ptr(rho), _ptr(drho), _ptr(full["aprior"]), 1):
            raise ValueError("oracle: id range beyond n")

    def set_schedule(self, t, tau, dt_ad, dt_ac, n_ac, n_adv, started):
        lib().osph_set_schedule(self._s, t, tau, dt_ad, dt_ac, int(n_ac), int(n_adv),
                                int(started))

    def sample_sigma(self, user_ids):
        ids = np.ascontiguousarray(user_ids, dtype=np.uint32)
        out = np.zeros(len(ids), np.float64)
        lib().osph_sample_sigma(self._s, len(ids), _ptr(ids), _ptr(out))
        return out
