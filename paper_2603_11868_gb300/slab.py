"""One tank decomposed into slabs along x over ranks.

The weakly-compressible SPH step of one tank shards by space: rank r owns the
fluid particles with x in [cut_r, cut_{r+1}) (the outer slabs open to -inf /
+inf) and holds, besides them, ghost copies of its neighbours' particles
within a halo of width W of its slab.  Each rank advances all of its
particles with the ordinary single-tank step (the library context, or any
engine with the same calls); a ghost's own update is not exact (its
neighbourhood is cut off at the halo's far side), so after every acoustic
step the owners send their exact state and the ghosts are overwritten:

  * the dependency radius of one acoustic step is four neighbour loops of 2h
    (density summation, viscous force, pressure and density relaxation) when
    it begins an advection step, two otherwise; a particle moves less than
    its drift budget (well under h) in an advection step.  W = 8h (4 cells)
    covers both, so every particle within reach of an owned particle's update
    is present on its rank with its exact state;
  * the ranks take one time step: after every step the squared velocity
    maximum over the owned particles is reduced (max) over the ranks and set
    in every engine, so every rank computes the same dt_ad, dt_ac and the
    same advection-step boundaries;
  * at every advection-step boundary (the next step rebuilds) ownership is
    decided again from the positions, which every rank holds exactly for its
    own and ghost particles: a particle that crossed a cut is already a ghost
    on the rank it moved to.  Each owner sends its new band particles (within
    W of a neighbour's slab) with their full state, and every rank loads its
    new set (owned, then ghosts) into its engine with the common schedule.

Local ids (the engine's user ids) are ordered
[sent to the left | interior | sent to the right | ghosts of the left
neighbour | ghosts of the right neighbour], so that the per-step exchange
moves contiguous id ranges.  A slab must be at least 2W wide (a particle is
never in both bands) and every rank must own particles.

Transport: SlabRank holds one rank's logic as phases; run_distributed drives
them with torch.distributed (gloo for host arrays, so the same path runs on
CPU ranks; the collectives are one scalar max per step and neighbour
exchanges of packed float64 arrays), run_in_process drives all ranks of a
group in one process (several engines on one device, one after the other:
nothing waits across ranks inside a kernel).
"""
from __future__ import annotations

import math

import numpy as np

HALO_CELLS = 4  # W in cells of 2h

STATE_KEYS = ("pos", "vel", "rho", "drho", "aprior")


def slab_cuts(x: np.ndarray, nranks: int, width: float) -> np.ndarray:
    """Cuts (nranks + 1 values, the outer ones infinite) that split the
    particles with x coordinates `x` into equal counts; interior cuts are
    spread to keep every slab at least `width` wide."""
    cuts = np.empty(nranks + 1)
    cuts[0], cuts[-1] = -math.inf, math.inf
    if nranks > 1:
        q = np.quantile(x, np.arange(1, nranks) / nranks)
        for k in range(1, nranks):
            lo = q[k - 1] if k == 1 else max(q[k - 1], cuts[k - 1] + width)
            cuts[k] = lo
    return cuts


def pack(gid: np.ndarray, st: dict, dim: int) -> np.ndarray:
    """(m, 3 dim + 3) float64 rows: gid, pos, vel, rho, drho, aprior."""
    m = len(gid)
    out = np.empty((m, 3 * dim + 3))
    out[:, 0] = gid
    out[:, 1:1 + dim] = st["pos"]
    out[:, 1 + dim:1 + 2 * dim] = st["vel"]
    out[:, 1 + 2 * dim] = st["rho"]
    out[:, 2 + 2 * dim] = st["drho"]
    out[:, 3 + 2 * dim:] = st["aprior"]
    return out


def unpack(rows: np.ndarray, dim: int):
    rows = rows.reshape(-1, 3 * dim + 3)
    st = {"pos": rows[:, 1:1 + dim], "vel": rows[:, 1 + dim:1 + 2 * dim],
          "rho": rows[:, 1 + 2 * dim], "drho": rows[:, 2 + 2 * dim],
          "aprior": rows[:, 3 + 2 * dim:]}
    return rows[:, 0].astype(np.int64), {k: np.ascontiguousarray(v) for k, v in st.items()}


def rows_of_state(st: dict, dim: int) -> np.ndarray:
    """(m, 3 dim + 2) float64 rows: pos, vel, rho, drho, aprior (the layout of
    the library's device rows)."""
    m = len(st["rho"])
    out = np.empty((m, 3 * dim + 2))
    out[:, :dim] = st["pos"]
    out[:, dim:2 * dim] = st["vel"]
    out[:, 2 * dim] = st["rho"]
    out[:, 2 * dim + 1] = st["drho"]
    out[:, 2 * dim + 2:] = st["aprior"]
    return out


def state_of_rows(rows: np.ndarray, dim: int) -> dict:
    rows = np.asarray(rows).reshape(-1, 3 * dim + 2)
    return {"pos": np.ascontiguousarray(rows[:, :dim]),
            "vel": np.ascontiguousarray(rows[:, dim:2 * dim]),
            "rho": np.ascontiguousarray(rows[:, 2 * dim]),
            "drho": np.ascontiguousarray(rows[:, 2 * dim + 1]),
            "aprior": np.ascontiguousarray(rows[:, 2 * dim + 2:])}


def _take(st: dict, idx) -> dict:
    return {k: np.ascontiguousarray(v[idx]) for k, v in st.items()}


def _cat(*parts: dict) -> dict:
    return {k: np.concatenate([p[k] for p in parts]) for k in STATE_KEYS}


class SlabRank:
    """One rank of a slab decomposition around an engine.

    The engine is anything with the calls set_state(state, sched) (load a new
    particle set, user ids 0..n-1 in the given order, with the schedule),
    get_state(id0, m), put_state(id0, state), step() (one acoustic step),
    schedule() / set_vmax2(v2) and owned_vmax2(n_own)."""

    def __init__(self, case, rank: int, nranks: int, engine, cuts=None,
                 halo_cells: int = HALO_CELLS):
        self.case, self.rank, self.nranks, self.engine = case, rank, nranks, engine
        self.dim = case.dim
        self.W = halo_cells * 2.0 * case.h
        x = case.fluid[:, 0]
        self.cuts = np.asarray(cuts) if cuts is not None else slab_cuts(x, nranks, 2 * self.W)
        widths = np.diff(self.cuts[1:-1]) if nranks > 2 else np.array([np.inf])
        if nranks > 2 and widths.min() < 2 * self.W:
            raise ValueError("slabs narrower than twice the halo")
        self.lo, self.hi = self.cuts[rank], self.cuts[rank + 1]
        # the initial particle set from the case (every rank holds the case)
        n = case.n
        vel = case.vel if case.vel is not None else np.zeros((n, self.dim))
        rho = case.rho if case.rho is not None else np.full(n, case.rho0)
        full = {"pos": case.fluid, "vel": vel, "rho": rho, "drho": np.zeros(n),
                "aprior": np.zeros((n, self.dim))}
        gid = np.arange(n)
        owner = np.searchsorted(self.cuts, x, side="right") - 1
        left_band = (owner == rank - 1) & (x >= self.lo - self.W)
        right_band = (owner == rank + 1) & (x < self.hi + self.W)
        self._load(gid, full, owner == rank, np.nonzero(left_band)[0],
                   np.nonzero(right_band)[0],
                   dict(t=0.0, tau=0.0, dt_ad=0.0, dt_ac=0.0, n_ac=0, n_adv=0, started=0,
                        vmax2=self._vmax2_of(vel)))

    @staticmethod
    def _vmax2_of(v: np.ndarray) -> float:
        if len(v) == 0:
            return 0.0
        s = v[:, 0] * v[:, 0] + v[:, 1] * v[:, 1]
        if v.shape[1] == 3:
            s = s + v[:, 2] * v[:, 2]
        return float(s.max())

    def _load(self, gid, st, own_mask, gl_idx, gr_idx, sched):
        """New local set: owned particles ordered [to left | interior | to right],
        then the ghosts of the left and of the right neighbour."""
        x = st["pos"][:, 0]
        own = np.nonzero(own_mask)[0]
        to_left = own[x[own] < self.lo + self.W] if self.rank > 0 else own[:0]
        to_right = own[x[own] >= self.hi - self.W] if self.rank < self.nranks - 1 else own[:0]
        if len(np.intersect1d(to_left, to_right)):
            raise ValueError("a particle lies in both bands of its slab")
        mid = np.setdiff1d(own, np.concatenate([to_left, to_right]), assume_unique=True)
        order = np.concatenate([to_left, mid, to_right, gl_idx, gr_idx]).astype(np.int64)
        self.n_own = len(own)
        if self.n_own == 0:
            raise ValueError(f"rank {self.rank} owns no particles")
        self.n_sl, self.n_sr = len(to_left), len(to_right)
        self.n_gl, self.n_gr = len(gl_idx), len(gr_idx)
        self.gid = np.asarray(gid)[order]
        self.engine.set_state(_take(st, order), sched)

    # -- phases ------------------------------------------------------------
    def needs_membership(self) -> bool:
        sc = self.engine.schedule()
        return bool(sc["started"]) and sc["tau"] >= sc["dt_ad"]

    def membership_outgoing(self):
        """The new owned particles in the bands of the neighbours, packed, and
        this rank's new owned set (kept for membership_apply)."""
        n = self.n_own + self.n_gl + self.n_gr
        st = self.engine.get_state(0, n)
        x = st["pos"][:, 0]
        owner = np.searchsorted(self.cuts, x, side="right") - 1
        mine = owner == self.rank
        self._pending = (self.gid.copy(), st, mine)
        out = []
        for nb, band in ((self.rank - 1, x < self.lo + self.W), (self.rank + 1, x >= self.hi - self.W)):
            if 0 <= nb < self.nranks:
                sel = np.nonzero(mine & band)[0]
                out.append(pack(self.gid[sel], _take(st, sel), self.dim))
            else:
                out.append(None)
        return out[0], out[1]

    def membership_apply(self, from_left, from_right):
        gid, st, mine = self._pending
        self._pending = None
        parts, gids = [_take(st, np.arange(len(gid)))], [gid]
        n0 = len(gid)
        idx = []
        for rows in (from_left, from_right):
            if rows is None or len(rows) == 0:
                idx.append(np.zeros(0, np.int64))
                continue
            g, s = unpack(rows, self.dim)
            idx.append(np.arange(n0, n0 + len(g)))
            n0 += len(g)
            parts.append(s)
            gids.append(g)
        allst, allgid = _cat(*parts), np.concatenate(gids)
        own_mask = np.zeros(len(allgid), bool)
        own_mask[:len(gid)] = mine
        sched = self.engine.schedule()
        self._load(allgid, allst, own_mask, idx[0], idx[1], sched)

    def step_local(self):
        self.engine.step()

    def local_vmax2(self) -> float:
        return self.engine.owned_vmax2(self.n_own)

    def set_global_vmax2(self, v2: float):
        self.engine.set_vmax2(v2)

    def _get_rows(self, id0, m):
        if hasattr(self.engine, "get_rows"):
            return self.engine.get_rows(id0, m)
        return rows_of_state(self.engine.get_state(id0, m), self.dim)

    def _put_rows(self, id0, rows):
        if hasattr(self.engine, "put_rows"):
            self.engine.put_rows(id0, rows)
        else:
            self.engine.put_state(id0, state_of_rows(rows, self.dim))

    def ghost_outgoing(self):
        """Rows of the owned particles in the neighbours' ghost bands (the
        order the neighbours hold them in since the last membership)."""
        to_l = self._get_rows(0, self.n_sl) if self.rank > 0 else None
        a = self.n_own - self.n_sr
        to_r = self._get_rows(a, self.n_sr) if self.rank < self.nranks - 1 else None
        return to_l, to_r

    def ghost_counts(self):
        """Rows this rank receives from its left and right neighbour."""
        return self.n_gl, self.n_gr

    def ghost_apply(self, from_left, from_right):
        for rows, id0, m in ((from_left, self.n_own, self.n_gl),
                             (from_right, self.n_own + self.n_gl, self.n_gr)):
            if m == 0:
                continue
            if rows is None or len(rows) != m:
                raise RuntimeError("ghost exchange out of step with the membership")
            self._put_rows(id0, rows)

    def owned_state(self):
        """(global ids, state) of the owned particles."""
        return self.gid[:self.n_own].copy(), self.engine.get_state(0, self.n_own)


def advance(ranks_or_rank, steps: int, exchange_packed, exchange_rows, allreduce_max):
    """Advance by `steps` acoustic steps.  For a list of this process's ranks:
    `exchange_packed(outgoing)` maps (to_left, to_right) packs per rank to
    (from_left, from_right) (the hand-over at advection-step boundaries, host
    arrays of unknown length); `exchange_rows(outgoing, counts)` does the same
    for the ghost rows, whose lengths every receiver knows; and
    `allreduce_max(values)` returns the maximum over all ranks."""
    ranks = ranks_or_rank if isinstance(ranks_or_rank, (list, tuple)) else [ranks_or_rank]
    for _ in range(steps):
        if ranks[0].needs_membership():
            got = exchange_packed([r.membership_outgoing() for r in ranks])
            for r, (fl, fr) in zip(ranks, got):
                r.membership_apply(fl, fr)
        for r in ranks:
            r.step_local()
        v2 = allreduce_max([r.local_vmax2() for r in ranks])
        for r in ranks:
            r.set_global_vmax2(v2)
        got = exchange_rows([r.ghost_outgoing() for r in ranks], [r.ghost_counts() for r in ranks])
        for r, (fl, fr) in zip(ranks, got):
            r.ghost_apply(fl, fr)


def _route(outs):
    res = []
    for k in range(len(outs)):
        fl = outs[k - 1][1] if k > 0 else None
        fr = outs[k + 1][0] if k + 1 < len(outs) else None
        res.append((fl, fr))
    return res


def _max_of(vals):
    if hasattr(vals[0], "view"):  # device scalars (torch): their elementwise maximum
        import torch
        out = vals[0].clone()
        for v in vals[1:]:
            out = torch.maximum(out, v)
        return out
    return max(vals)


def run_in_process(ranks, steps: int):
    """All ranks of a group in one process: exchanges route the arrays
    between the rank objects directly."""
    advance(list(ranks), steps, _route, lambda outs, counts: _route(outs), _max_of)


def run_distributed(rank_obj: SlabRank, steps: int, dist, device="cpu"):
    """One rank per process over torch.distributed: the hand-over packs as
    point-to-point messages (length, then rows) through `device` (cpu for
    gloo, the rank's GPU for nccl); the ghost rows as point-to-point messages
    of known length (device tensors when the engine keeps them on the device);
    the velocity maximum as an all-reduce (max of the 64-bit patterns of
    non-negative doubles, which order like the values)."""
    import torch
    r, n = rank_obj.rank, rank_obj.nranks
    nbs = [(r - 1, 0), (r + 1, 1)]

    def exchange_packed(outs):
        out = outs[0]
        reqs, lens = [], {}
        for nb, side in nbs:
            if 0 <= nb < n:
                arr = out[side]
                t = torch.tensor([0 if arr is None else arr.shape[0]], dtype=torch.int64,
                                 device=device)
                reqs.append(dist.isend(t, nb))
                lens[nb] = torch.zeros(1, dtype=torch.int64, device=device)
                reqs.append(dist.irecv(lens[nb], nb))
        for q in reqs:
            q.wait()
        width = 3 * rank_obj.dim + 3
        reqs, bufs, keep = [], {}, []
        for nb, side in nbs:
            if 0 <= nb < n:
                arr = out[side]
                if arr is not None and arr.shape[0] > 0:
                    t = torch.from_numpy(np.ascontiguousarray(arr)).to(device)
                    keep.append(t)
                    reqs.append(dist.isend(t, nb))
                m = int(lens[nb].item())
                bufs[nb] = torch.empty((m, width), dtype=torch.float64, device=device)
                if m > 0:
                    reqs.append(dist.irecv(bufs[nb], nb))
        for q in reqs:
            q.wait()
        got = [bufs[nb].cpu().numpy() if nb in bufs else None for nb, _ in nbs]
        return [(got[0], got[1])]

    def exchange_rows(outs, counts):
        out, cnt = outs[0], counts[0]
        width = 3 * rank_obj.dim + 2
        reqs, got, keep = [], [None, None], []
        for nb, side in nbs:
            if not 0 <= nb < n:
                continue
            arr = out[side]
            if arr is not None and len(arr) > 0:
                t = arr if torch.is_tensor(arr) else torch.from_numpy(
                    np.ascontiguousarray(arr)).to(device)
                keep.append(t)
                reqs.append(dist.isend(t, nb))
            m = cnt[side]
            # received where the engine keeps its rows (the sent rows' device)
            buf = torch.empty((m, width), dtype=torch.float64,
                              device=arr.device if torch.is_tensor(arr) else device)
            if m > 0:
                reqs.append(dist.irecv(buf, nb))
            got[side] = buf
        for q in reqs:
            q.wait()
        return [tuple(g if g is None or g.device.type != "cpu" else g.numpy() for g in got)]

    def allreduce_max(vals):
        v = vals[0]
        if torch.is_tensor(v):
            bits = v.view(torch.int64)
            dist.all_reduce(bits, op=dist.ReduceOp.MAX)
            return bits.view(torch.float64)
        t = torch.tensor([v], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    advance(rank_obj, steps, exchange_packed, exchange_rows, allreduce_max)


class LibraryEngine:
    """The CUDA library's context as a slab engine.  The hand-over at
    advection-step boundaries moves host arrays; with device_rows the per-step
    ghost rows and the velocity maximum stay in device memory (torch tensors
    on the current stream, which the library's calls are ordered with)."""

    def __init__(self, case, precision: str = "mixed", walls=None, wall_vel=None,
                 device_rows: bool = False):
        self.device_rows = device_rows
        from . import sph
        self.sph = sph
        self.case = case
        self.dim = case.dim
        self.precision = sph.SPH_FP64 if precision == "fp64" else sph.SPH_MIXED
        self._allocator = sph.TorchAllocator()
        import torch
        stream = torch.cuda.current_stream().cuda_stream
        self.ctx = sph.sph_create(case.dim, case.lo, case.hi, case.dp, case.h, case.rho0,
                                  case.c0, case.mu, case.U_ref, case.gravity, self.precision,
                                  self._allocator.struct, stream)
        w = case.wall if walls is None else walls
        if w is not None and len(w):
            sph.sph_set_particles(self.ctx, sph.SPH_WALL, w, wall_vel)
        self.n = 0

    def set_state(self, st, sched):
        sph = self.sph
        self.n = len(st["rho"])
        sph.sph_set_particles(self.ctx, sph.SPH_FLUID, st["pos"], st["vel"], st["rho"])
        sph.sph_put_state_range(self.ctx, 0, {"drho": st["drho"], "aprior": st["aprior"]})
        sph.sph_set_schedule(self.ctx, sched)

    def get_state(self, id0, m):
        return self.sph.sph_get_state_range(self.ctx, id0, m, self.dim)

    def put_state(self, id0, st):
        self.sph.sph_put_state_range(self.ctx, id0, st)

    def step(self):
        self.sph.sph_step(self.ctx, 1)

    def schedule(self):
        return self.sph.sph_get_schedule(self.ctx)

    def owned_vmax2(self, n_own):
        if not self.device_rows:
            return self.sph.sph_owned_vmax2(self.ctx, n_own)
        import torch
        t = torch.empty(1, dtype=torch.float64, device="cuda")
        self.sph._check(self.ctx, self.sph.load().sph_owned_vmax2_device(self.ctx, int(n_own),
                                                                         t.data_ptr()))
        return t

    def set_vmax2(self, v2):
        if hasattr(v2, "data_ptr"):
            self.sph._check(self.ctx, self.sph.load().sph_set_vmax2_device(self.ctx,
                                                                           v2.data_ptr()))
        else:
            self.sph.sph_set_vmax2(self.ctx, v2)

    def get_rows(self, id0, m):
        if not self.device_rows:
            return rows_of_state(self.get_state(id0, m), self.dim)
        import torch
        t = torch.empty((m, 3 * self.dim + 2), dtype=torch.float64, device="cuda")
        self.sph._check(self.ctx, self.sph.load().sph_get_state_rows_device(
            self.ctx, int(id0), int(m), t.data_ptr()))
        return t

    def put_rows(self, id0, rows):
        if hasattr(rows, "data_ptr"):
            rows = rows.contiguous()
            self.sph._check(self.ctx, self.sph.load().sph_put_state_rows_device(
                self.ctx, int(id0), int(rows.shape[0]), rows.data_ptr()))
        else:
            self.put_state(id0, state_of_rows(rows, self.dim))

    def close(self):
        if getattr(self, "ctx", None):
            self.sph.sph_destroy(self.ctx)
            self.ctx = None
