// Neighbour search on the device: cell keys, stable LSD radix sort, CSR cell
// offsets; plus the schedule control kernel, the velocity maximum and the
// neighbour-set fingerprint used by parity checks.
//
// The paper bins particles into cells of the cut-off size for its cell-linked
// list and sorts particles on the device with a radix sort instead of the CPU
// quick sort (section "Cell linked-list, direct search and sorting").  Here the
// linked list is replaced by a sort-based CSR structure: key -> stable sort ->
// per-cell [begin, end) offsets.  It is deterministic (no atomics decide an
// order), so keys, permutation and offsets are bit-identical to a serial
// stable sort.
#include "sph_internal.cuh"

namespace sphgb {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

struct XSet {
  const double* x[2][3];
};

__global__ void k_cell_keys(Params P, XSet xs, uint32_t* __restrict__ keys,
                            uint32_t* __restrict__ vals, int n, DevScalars* sc, int gated,
                            uint32_t* digit_total, int bins) {
  if (gated && !sc->new_adv) return;
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < bins; t += blockDim.x) digit_total[t] = 0;
  const int par = sc ? sc->par : 0;
  const double* __restrict__ x0 = xs.x[par][0];
  const double* __restrict__ x1 = xs.x[par][1];
  const double* __restrict__ x2 = xs.x[par][2];
  int oob = 0;
  const float inv_cs = (float)(1.0 / P.cs);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int cx = cell_coord_fast(x0[i], P.lo[0], P.cs, inv_cs, P.nx, oob);
    int cy = cell_coord_fast(x1[i], P.lo[1], P.cs, inv_cs, P.ny, oob);
    int cz = P.dim == 3 ? cell_coord_fast(x2[i], P.lo[2], P.cs, inv_cs, P.nz, oob) : 0;
    keys[i] = ((uint32_t)cz * (uint32_t)P.ny + (uint32_t)cy) * (uint32_t)P.nx + (uint32_t)cx;
    vals[i] = (uint32_t)i;
  }
  if (__syncthreads_or(oob) && threadIdx.x == 0 && sc) atomicOr(&sc->flags, kFlagOutOfDomain);
}

// ---------------------------------------------------------------------------
// Radix sort, one pass = histogram, scan, scatter.  A tile is kSortTile keys;
// warp w of a block owns the contiguous slice [w*32*kSortItems, ...) of its
// tile and walks it in rounds of 32, so processing order = input order and
// ranks are stable.  Histograms and ranks use __match_any_sync: the lanes that
// share a digit count once per round through their leader.

// The key count is n, or *n_dev when n_dev is given (a count decided on the
// device; the grid is then sized for n, its upper bound).
__device__ __forceinline__ void sort_count(int& n, int& tiles, const int* n_dev) {
  if (n_dev) {
    n = *n_dev;
    tiles = (n + kSortTile - 1) / kSortTile;
  }
}

// Lanes holding the same digit (a valid lane's d < 2^nbits): one ballot per
// digit bit and one for validity, ANDed; the same mask as __match_any_sync on
// (valid, d), from full-rate instructions.
__device__ __forceinline__ unsigned match_digit(uint32_t d, bool valid, int nbits) {
  const unsigned vb = __ballot_sync(kFull, valid);
  unsigned m = valid ? vb : ~vb;
  for (int b = 0; b < nbits; ++b) {
    const bool bit = (d >> b) & 1u;
    const unsigned bb = __ballot_sync(kFull, bit);
    m &= bit ? bb : ~bb;
  }
  return m;
}

// kBallot: equal digits grouped by match_digit (measured faster for keys in
// random order: a warp then holds many distinct digits), else by
// __match_any_sync (faster for the nearly sorted keys of a re-sort).
template <bool kBallot>
__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int n, int shift, uint32_t mask,
                             uint32_t* __restrict__ tile_hist, uint32_t* digit_total, int tiles,
                             const DevScalars* sc, int gated, const int* n_dev) {
  if (gated && !sc->new_adv) return;
  sort_count(n, tiles, n_dev);
  if ((int)blockIdx.x >= tiles) return;
  extern __shared__ uint32_t smem[];
  const int bins = (int)mask + 1;
  const int warps = blockDim.x / 32;
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  uint32_t* wh = smem;  // [warps][bins]
  for (int t = threadIdx.x; t < warps * bins; t += blockDim.x) wh[t] = 0;
  __syncthreads();
  const int tile = blockIdx.x;
  const long base = (long)tile * kSortTile + (long)w * 32 * kSortItems;
#pragma unroll 4
  for (int it = 0; it < kSortItems; ++it) {
    long idx = base + it * 32 + lane;
    bool valid = idx < n;
    unsigned peers;
    uint32_t d;
    if constexpr (kBallot) {
      d = valid ? (keys[idx] >> shift) & mask : 0u;
      peers = match_digit(d, valid, __popc(mask));
    } else {
      d = valid ? (keys[idx] >> shift) & mask : 0xffffffffu;
      peers = __match_any_sync(kFull, d);
    }
    if (valid && lane == __ffs(peers) - 1) wh[w * bins + d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  for (int d = threadIdx.x; d < bins; d += blockDim.x) {
    uint32_t s = 0;
    for (int q = 0; q < warps; ++q) s += wh[q * bins + d];
    tile_hist[(long)d * tiles + tile] = s;
    if (s) atomicAdd(&digit_total[d], s);
  }
}

// Block-wide exclusive scan of one value per thread (256 threads).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums,
                                                         uint32_t& total) {
  const int lane = threadIdx.x % 32, w = threadIdx.x / 32, warps = blockDim.x / 32;
  uint32_t incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[w] = incl;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < warps ? warp_sums[lane] : 0;
    uint32_t si = s;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(kFull, si, o);
      if (lane >= o) si += t;
    }
    if (lane < warps) warp_sums[lane] = si - s;  // exclusive prefix of warp totals
    if (lane == warps - 1) warp_sums[32] = si;
  }
  __syncthreads();
  uint32_t r = warp_sums[w] + incl - v;
  total = warp_sums[32];
  __syncthreads();
  return r;
}

// One block per digit: offsets[d][t] = sum of all digits < d + sum of tiles < t.
__global__ void k_radix_scan(uint32_t* __restrict__ tile_hist, const uint32_t* digit_total,
                             int tiles, const DevScalars* sc, int gated, const int* n_dev) {
  if (gated && !sc->new_adv) return;
  int n = 0;
  sort_count(n, tiles, n_dev);
  __shared__ uint32_t ws[33];
  const int d = blockIdx.x;
  uint32_t part = 0;
  for (int q = threadIdx.x; q < d; q += blockDim.x) part += digit_total[q];
  uint32_t tot;
  block_exclusive_scan(part, ws, tot);
  const uint32_t base = tot;
  const int per = (tiles + blockDim.x - 1) / blockDim.x;
  const int t0 = threadIdx.x * per;
  uint32_t* row = tile_hist + (long)d * tiles;
  uint32_t s = 0;
  for (int t = t0; t < t0 + per && t < tiles; ++t) s += row[t];
  uint32_t dummy;
  uint32_t run = base + block_exclusive_scan(s, ws, dummy);
  for (int t = t0; t < t0 + per && t < tiles; ++t) {
    uint32_t c = row[t];
    row[t] = run;
    run += c;
  }
}

__global__ void k_radix_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, int n,
                                int shift, uint32_t mask, const uint32_t* __restrict__ offsets,
                                int tiles, const DevScalars* sc, int gated,
                                uint32_t* digit_total, const int* n_dev) {
  if (gated && !sc->new_adv) return;
  sort_count(n, tiles, n_dev);
  extern __shared__ uint32_t smem[];
  const int bins = (int)mask + 1;
  const int warps = blockDim.x / 32;
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  uint32_t* wcnt = smem;                       // [warps][bins]
  uint32_t* lbase = wcnt + warps * bins;       // [bins] local (tile) start of each digit
  uint32_t* goff = lbase + bins;               // [bins] global start of each digit
  uint32_t* skey = goff + bins;                // [kSortTile]
  uint32_t* sval = skey + kSortTile;           // [kSortTile]
  __shared__ uint32_t ws[33];
  if (blockIdx.x == 0) {
    // the scan of this pass has consumed the totals: clear them for the next pass
    for (int t = threadIdx.x; t < bins; t += blockDim.x) digit_total[t] = 0;
  }
  if ((int)blockIdx.x >= tiles) return;
  for (int t = threadIdx.x; t < warps * bins; t += blockDim.x) wcnt[t] = 0;
  __syncthreads();
  const int tile = blockIdx.x;
  const long base = (long)tile * kSortTile + (long)w * 32 * kSortItems;
  uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    long idx = base + it * 32 + lane;
    bool valid = idx < n;
    key[it] = valid ? kin[idx] : 0u;
    val[it] = valid ? vin[idx] : 0u;
    uint32_t d = valid ? (key[it] >> shift) & mask : 0xffffffffu;
    unsigned peers = __match_any_sync(kFull, d);
    uint32_t cnt = valid ? wcnt[w * bins + d] : 0u;
    rank[it] = cnt + __popc(peers & lanemask_lt());
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[w * bins + d] = cnt + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, block totals -> local starts
  const int per = (bins + blockDim.x - 1) / blockDim.x;
  uint32_t tot_local = 0;
  for (int q = 0; q < per; ++q) {
    int d = threadIdx.x * per + q;
    if (d < bins) {
      uint32_t run = 0;
      for (int ww = 0; ww < warps; ++ww) {
        uint32_t t = wcnt[ww * bins + d];
        wcnt[ww * bins + d] = run;
        run += t;
      }
      lbase[d] = run;  // digit total for now
      tot_local += run;
    }
  }
  uint32_t tall;
  uint32_t start = block_exclusive_scan(tot_local, ws, tall);
  for (int q = 0; q < per; ++q) {
    int d = threadIdx.x * per + q;
    if (d < bins) {
      uint32_t c = lbase[d];
      lbase[d] = start;
      start += c;
      goff[d] = offsets[(long)d * tiles + tile];
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    long idx = base + it * 32 + lane;
    if (idx < n) {
      uint32_t d = (key[it] >> shift) & mask;
      uint32_t pos = lbase[d] + wcnt[w * bins + d] + rank[it];
      skey[pos] = key[it];
      sval[pos] = val[it];
    }
  }
  __syncthreads();
  const long tile0 = (long)tile * kSortTile;
  const int cnt = (int)min((long)kSortTile, (long)n - tile0);
  for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
    uint32_t k = skey[q];
    uint32_t d = (k >> shift) & mask;
    uint32_t g = goff[d] + (uint32_t)q - lbase[d];
    kout[g] = k;
    vout[g] = sval[q];
  }
}

// ---------------------------------------------------------------------------
// First index in sorted keys[0..n) whose key is >= c (32-ary search by one warp).
__device__ uint32_t warp_lower_bound(const uint32_t* __restrict__ keys, uint32_t n, uint32_t c) {
  const int lane = threadIdx.x % 32;
  uint32_t a = 0, b = n;
  while (b - a > 32) {
    uint32_t len = b - a;
    uint32_t idx = a + (uint32_t)(((unsigned long long)len * (lane + 1)) / 33);
    bool pred = keys[idx] < c;
    unsigned bal = __ballot_sync(kFull, pred);
    int cntp = __popc(bal);
    uint32_t lo_idx = __shfl_sync(kFull, idx, cntp > 0 ? cntp - 1 : 0);
    uint32_t hi_idx = __shfl_sync(kFull, idx, cntp < 32 ? cntp : 31);
    if (cntp > 0) a = lo_idx + 1;
    if (cntp < 32) b = hi_idx;
  }
  bool pred = (a + lane < b) && keys[a + lane] < c;
  return a + __popc(__ballot_sync(kFull, pred));
}

// Offsets of the local cells [c0, c1) of one grid whose sorted keys are
// keys[0..n) (key = kbase + local cell): cb[c] = first + (first position with
// key >= kbase + c); the chunk that ends at ncell also writes cb[ncell] =
// first + n.  One block per chunk; blocks may call it for several chunks.
__device__ __forceinline__ void offsets_chunk(const uint32_t* __restrict__ keys, uint32_t n,
                                              uint32_t kbase, uint32_t c0, uint32_t c1,
                                              uint32_t ncell, uint32_t first,
                                              uint32_t* __restrict__ cb) {
  __shared__ uint32_t sfirst[kOffsetsChunk];
  __shared__ uint32_t bounds[2];
  __shared__ uint32_t wmin[32];
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (w < 2) {
    uint32_t r = warp_lower_bound(keys, n, kbase + (w == 0 ? c0 : c1));
    if (lane == 0) bounds[w] = r;
  }
  __syncthreads();
  const uint32_t lo = bounds[0], hi = bounds[1];
  for (int t = threadIdx.x; t < kOffsetsChunk; t += blockDim.x) sfirst[t] = hi;
  __syncthreads();
  for (uint32_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
    uint32_t kk = keys[k];
    if (k == lo || keys[k - 1] != kk) sfirst[kk - kbase - c0] = k;
  }
  __syncthreads();
  // suffix minimum: an empty cell starts where the next non-empty cell starts
  constexpr int PER = kOffsetsChunk / 256;
  uint32_t v[PER];
  const int t0 = threadIdx.x * PER;
#pragma unroll
  for (int j = 0; j < PER; ++j) v[j] = sfirst[t0 + j];
#pragma unroll
  for (int j = PER - 2; j >= 0; --j) v[j] = min(v[j], v[j + 1]);
  uint32_t incl = v[0];
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_down_sync(kFull, incl, o);
    if (lane + o < 32) incl = min(incl, t);
  }
  if (lane == 0) wmin[w] = incl;
  __syncthreads();
  uint32_t carry = 0xffffffffu;
  for (int q = w + 1; q < (int)(blockDim.x / 32); ++q) carry = min(carry, wmin[q]);
  uint32_t right = __shfl_down_sync(kFull, incl, 1);
  if (lane == 31) right = 0xffffffffu;
  uint32_t excl = min(right, carry);
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    uint32_t c = c0 + t0 + j;
    if (c < c1) cb[c] = first + min(v[j], excl);
  }
  if (c1 == ncell && threadIdx.x == 0) cb[ncell] = first + n;
  __syncthreads();  // the shared arrays are reused by the block's next chunk
}

// cell_begin of one grid, kOffsetsChunk cells per block (256 threads).
__global__ void k_cell_offsets(const uint32_t* __restrict__ keys, int n, uint32_t ncell,
                               uint32_t* __restrict__ cb, DevScalars* sc, int gated,
                               int flip_par) {
  if (gated && !sc->new_adv) return;
  const uint32_t c0 = blockIdx.x * kOffsetsChunk;
  const uint32_t c1 = min(c0 + (uint32_t)kOffsetsChunk, ncell);
  offsets_chunk(keys, (uint32_t)n, 0u, c0, c1, ncell, 0u, cb);
  if (flip_par && blockIdx.x == 0 && threadIdx.x == 0) sc->par ^= 1;
}

// ---------------------------------------------------------------------------
// Dual-criteria schedule, one thread.  vmax2_cur holds max |v|^2 of the
// current velocities.  At an advection step it also sizes the skin (the cap
// of the particles' drift budgets) and clears the lists' validity flags.
__device__ __forceinline__ void control_one(const Params& P, DevScalars* sc) {
  double vmax = sqrt(__longlong_as_double((long long)sc->vmax2_cur));
  int adv = (!sc->started || sc->tau >= sc->dt_ad) ? 1 : 0;
  double dt = 0.6 * P.h / (P.c0 + vmax);
  if (adv) {
    sc->dt_ad = 0.25 * P.h / (P.U_ref > vmax ? P.U_ref : vmax);
    sc->tau = 0.0;
    sc->n_adv += 1;
    sc->started = 1;
    // skin for this advection step: twice the distance covered at the current
    // top speed (plus what gravity can add; at least the speed of a
    // translating wall) over the step and one overshooting acoustic step, with
    // margin; no particle's drift budget exceeds half of it
    const double gmag = sqrt(P.g[0] * P.g[0] + P.g[1] * P.g[1] + P.g[2] * P.g[2]);
    const double span = sc->dt_ad + 1.5 * dt;
    const double vs = vmax > P.wall_vmax ? vmax : P.wall_vmax;
    double skin = 2.5 * (vs + gmag * span) * span + 0.02 * P.h;
    sc->skin = skin < P.skin_max ? skin : P.skin_max;
    sc->list_bad = 0;
    sc->t_reb = sc->t;
    // per-particle drift budgets are set by the reorder from each particle's
    // speed; walls all get the translating walls' one
    sc->drift_bad_p = 0;
    sc->drift_bad_r = 0;
    sc->wall_budget = 1.25 * P.wall_vmax * span;
  }
  sc->new_adv = adv;
  sc->dt_ac = dt;
  sc->tau += dt;
  sc->t0 = sc->t;
  sc->t += dt;
  sc->n_ac += 1;
  sc->vmax2_next = 0ull;
}

// use_cond: the step runs as a CUDA graph whose rebuild stages sit in a
// conditional node; the schedule's decision opens or skips it on the device.
__global__ void k_control(Params P, DevScalars* sc, cudaGraphConditionalHandle cond,
                          int use_cond) {
  control_one(P, sc);
  if (use_cond) cudaGraphSetConditional(cond, sc->new_adv ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Batched schedule: one thread per tank (one block of up to kMaxTanks
// threads).  The velocity maximum of the previous step's pressure stage
// becomes the current one, the tank's schedule advances as for a single tank,
// and the tanks that begin an advection step are listed (in tank order) with
// their tile, chunk and compacted-slot prefixes.
__global__ void kb_control(BatchArgs A, int tile, int force) {
  __shared__ uint32_t ws[33];
  WorkList* wl = A.wl_adv;
  const int t = threadIdx.x;
  uint32_t on = 0, tiles = 0, chunks = 0, n = 0;
  if (t < A.ntanks) {
    const Params& P = A.tP[t];
    DevScalars* sc = A.tsc + t;
    if (force) {
      on = 1;
    } else {
      if (sc->started) sc->vmax2_cur = sc->vmax2_next;
      control_one(P, sc);
      on = sc->new_adv && P.n > 0;
    }
    if (on) {
      n = (uint32_t)P.n;
      tiles = (n + (uint32_t)tile - 1) / (uint32_t)tile;
      chunks = (P.ncell + kOffsetsChunk - 1) / kOffsetsChunk;
    }
  }
  uint32_t tot_on, tot_tiles, tot_chunks, tot_n;
  const uint32_t pos = block_exclusive_scan(on, ws, tot_on);
  const uint32_t tp = block_exclusive_scan(tiles, ws, tot_tiles);
  const uint32_t cp = block_exclusive_scan(chunks, ws, tot_chunks);
  const uint32_t np = block_exclusive_scan(n, ws, tot_n);
  if (on) {
    wl->tank[pos] = t;
    wl->tile_prefix[pos] = (int)tp;
    wl->chunk_prefix[pos] = (int)cp;
    wl->cbase[pos] = (int)np;
  }
  if (t == 0) {
    wl->count = (int)tot_on;
    wl->tiles = (int)tot_tiles;
    wl->chunks = (int)tot_chunks;
    wl->m = (int)tot_n;
    wl->tile = tile;
    wl->tile_prefix[tot_on] = (int)tot_tiles;
    wl->chunk_prefix[tot_on] = (int)tot_chunks;
  }
}

// Batched cell keys: slot first + q of a listed tank goes to compacted slot
// cbase + q with key cell_base + (its cell in the tank's grid), value = slot.
__global__ void kb_cell_keys(BatchArgs A, const WorkList* wl, int walls, XSet xs,
                             uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                             uint32_t* digit_total, int bins) {
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < bins; t += blockDim.x) digit_total[t] = 0;
  for_each_tile(wl, [&](int a, int off, int tile) {
    const int t = wl->tank[a];
    const Params& P = A.tP[t];
    const int par = walls ? 0 : A.tsc[t].par;
    const int first = walls ? P.woff : P.foff, cnt = walls ? P.nw : P.n;
    const int base = wl->cbase[a];
    const double* __restrict__ x0 = par ? xs.x[1][0] : xs.x[0][0];
    const double* __restrict__ x1 = par ? xs.x[1][1] : xs.x[0][1];
    const double* __restrict__ x2 = par ? xs.x[1][2] : xs.x[0][2];
    const float inv_cs = (float)(1.0 / P.cs);
    const double lo0 = P.lo[0], lo1 = P.lo[1], lo2 = P.lo[2], cs = P.cs;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const uint32_t cbase = P.cell_base;
    int oob = 0;
    const int end = min(off + tile, cnt);
    for (int q = off + (int)threadIdx.x; q < end; q += blockDim.x) {
      const int i = first + q;
      const int cx = cell_coord_fast(x0[i], lo0, cs, inv_cs, nx, oob);
      const int cy = cell_coord_fast(x1[i], lo1, cs, inv_cs, ny, oob);
      const int cz = P.dim == 3 ? cell_coord_fast(x2[i], lo2, cs, inv_cs, nz, oob) : 0;
      keys[base + q] =
          cbase + ((uint32_t)cz * (uint32_t)ny + (uint32_t)cy) * (uint32_t)nx + (uint32_t)cx;
      vals[base + q] = (uint32_t)i;
    }
    if (__syncthreads_or(oob) && threadIdx.x == 0 && !walls)
      atomicOr(&A.tsc[t].flags, kFlagOutOfDomain);
  });
}

// Batched CSR offsets of the listed tanks (chunks of kOffsetsChunk cells);
// flip_par: the tank's live copy flips once its reorder is done.
__global__ void kb_cell_offsets(BatchArgs A, const WorkList* wl, int walls,
                                const uint32_t* __restrict__ keys, uint32_t* cb, int flip_par) {
  for_each_chunk(wl, [&](int a, int j) {
    const int t = wl->tank[a];
    const Params& P = A.tP[t];
    const uint32_t n = (uint32_t)(walls ? P.nw : P.n);
    const uint32_t first = (uint32_t)(walls ? P.woff : P.foff);
    const uint32_t ncell = P.ncell, kbase = P.cell_base;
    const uint32_t c0 = (uint32_t)j * kOffsetsChunk;
    const uint32_t c1 = min(c0 + (uint32_t)kOffsetsChunk, ncell);
    offsets_chunk(keys + wl->cbase[a], n, kbase, c0, c1, ncell, first, cb + kbase);
    if (flip_par && j == 0 && threadIdx.x == 0) A.tsc[t].par ^= 1;
  });
}

// |v|^2 without contraction, same rounding sequence as a plain serial sum
__device__ __forceinline__ double speed2(double a, double b, double c) {
  return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}

__global__ void k_vmax(Params P, DevBuffers B, int n) {
  DevScalars* sc = B.sc;
  const int par = sc->par;
  const double* v0 = B.v[par][0];
  const double* v1 = B.v[par][1];
  const double* v2 = B.v[par][2];
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = speed2(v0[i], v1[i], P.dim == 3 ? v2[i] : 0.0);
    m = s > m ? s : m;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
  __shared__ double wm[32];
  if (threadIdx.x % 32 == 0) wm[threadIdx.x / 32] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x / 32); ++q) m = fmax(m, wm[q]);
    atomicMax(&sc->vmax2_cur, (unsigned long long)__double_as_longlong(m));
  }
}

// Per-particle state of the particles with user ids [id0, id0 + m) (the
// live copy): gather into / scatter from arrays in user-id order, `comps`
// values per particle (field: 0 position, 1 velocity, 2 density, 3 density
// rate, 4 prior acceleration; the last two in the pair type).
__global__ void k_state_range(Params P, DevBuffers B, uint32_t id0, uint32_t m, double* buf,
                              int field, int put, int pair_is_float) {
  DevScalars* sc = B.sc;
  const int par = sc->par;
  const uint32_t* id = B.id[par];
  const int d = P.dim;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.n; s += gridDim.x * blockDim.x) {
    const uint32_t u = id[s] - id0;
    if (u >= m) continue;
    switch (field) {
      case 0:
      case 1:
        for (int k = 0; k < d; ++k) {
          double* a = field == 0 ? B.x[par][k] : B.v[par][k];
          if (put) a[s] = buf[(size_t)u * d + k]; else buf[(size_t)u * d + k] = a[s];
        }
        break;
      case 2:
        if (put) B.rho[par][s] = buf[u]; else buf[u] = B.rho[par][s];
        break;
      case 3:
        if (pair_is_float) {
          float* a = (float*)B.drho[par];
          if (put) a[s] = (float)buf[u]; else buf[u] = a[s];
        } else {
          double* a = (double*)B.drho[par];
          if (put) a[s] = buf[u]; else buf[u] = a[s];
        }
        break;
      default:
        for (int k = 0; k < d; ++k) {
          if (pair_is_float) {
            float* a = (float*)B.aprior[k];
            if (put) a[s] = (float)buf[(size_t)u * d + k]; else buf[(size_t)u * d + k] = a[s];
          } else {
            double* a = (double*)B.aprior[k];
            if (put) a[s] = buf[(size_t)u * d + k]; else buf[(size_t)u * d + k] = a[s];
          }
        }
    }
  }
}

// The state of user ids [id0, id0 + m) as packed rows in user-id order,
// 3 dim + 2 doubles each: position, velocity, density, density rate, prior
// acceleration; gathered into (put = 0) or scattered from (put = 1) rows.
__global__ void k_state_rows(Params P, DevBuffers B, uint32_t id0, uint32_t m, double* rows,
                             int put, int pair_is_float) {
  DevScalars* sc = B.sc;
  const int par = sc->par;
  const uint32_t* id = B.id[par];
  const int d = P.dim, w = 3 * d + 2;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < P.n; s += gridDim.x * blockDim.x) {
    const uint32_t u = id[s] - id0;
    if (u >= m) continue;
    double* r = rows + (size_t)u * w;
    for (int k = 0; k < d; ++k) {
      if (put) {
        B.x[par][k][s] = r[k];
        B.v[par][k][s] = r[d + k];
      } else {
        r[k] = B.x[par][k][s];
        r[d + k] = B.v[par][k][s];
      }
    }
    if (put) B.rho[par][s] = r[2 * d]; else r[2 * d] = B.rho[par][s];
    if (pair_is_float) {
      float* dr = (float*)B.drho[par];
      if (put) dr[s] = (float)r[2 * d + 1]; else r[2 * d + 1] = dr[s];
      for (int k = 0; k < d; ++k) {
        float* a = (float*)B.aprior[k];
        if (put) a[s] = (float)r[2 * d + 2 + k]; else r[2 * d + 2 + k] = a[s];
      }
    } else {
      double* dr = (double*)B.drho[par];
      if (put) dr[s] = r[2 * d + 1]; else r[2 * d + 1] = dr[s];
      for (int k = 0; k < d; ++k) {
        double* a = (double*)B.aprior[k];
        if (put) a[s] = r[2 * d + 2 + k]; else r[2 * d + 2 + k] = a[s];
      }
    }
  }
}

// max |v|^2 over the particles with user ids below n_own (the live copy)
__global__ void k_vmax_owned(Params P, DevBuffers B, uint32_t n_own, unsigned long long* out) {
  DevScalars* sc = B.sc;
  const int par = sc->par;
  const uint32_t* id = B.id[par];
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    if (id[i] >= n_own) continue;
    const double s = speed2(B.v[par][0][i], B.v[par][1][i], P.dim == 3 ? B.v[par][2][i] : 0.0);
    m = s > m ? s : m;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

__global__ void kb_vmax(BatchArgs A, DevBuffers B) {
  __shared__ double wm[32];
  const WorkList* wl = A.wl_all;
  for_each_tile(wl, [&](int a, int off, int tile) {
    const int t = wl->tank[a];
    const Params& P = A.tP[t];
    const int par = A.tsc[t].par;
    const double* v0 = par ? B.v[1][0] : B.v[0][0];
    const double* v1 = par ? B.v[1][1] : B.v[0][1];
    const double* v2 = par ? B.v[1][2] : B.v[0][2];
    const int end = min(off + tile, P.n);
    double m = 0.0;
    for (int q = off + (int)threadIdx.x; q < end; q += blockDim.x) {
      const int i = P.foff + q;
      const double s = speed2(v0[i], v1[i], P.dim == 3 ? v2[i] : 0.0);
      m = s > m ? s : m;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
    __syncthreads();
    if (threadIdx.x % 32 == 0) wm[threadIdx.x / 32] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int q = 1; q < (int)(blockDim.x / 32); ++q) m = fmax(m, wm[q]);
      atomicMax(&A.tsc[t].vmax2_cur, (unsigned long long)__double_as_longlong(m));
    }
  });
}

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double dist2_exact(double ax, double ay, double az, double bx, double by,
                                              double bz) {
  double d0 = __dsub_rn(ax, bx), d1 = __dsub_rn(ay, by), d2 = __dsub_rn(az, bz);
  return __dadd_rn(__dadd_rn(__dmul_rn(d0, d0), __dmul_rn(d1, d1)), __dmul_rn(d2, d2));
}

__global__ void k_neighbour_stats(Params P, DevBuffers B, const double* __restrict__ wx,
                                  const double* __restrict__ wy, const double* __restrict__ wz,
                                  uint32_t* cnt_f, uint32_t* cnt_w, unsigned long long* hash) {
  const int par = B.sc->par;
  const double* x0 = B.x[par][0];
  const double* x1 = B.x[par][1];
  const double* x2 = B.x[par][2];
  const uint32_t* keys = B.keys[B.sorted_buf];
  const uint32_t* id = B.id[par];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    uint32_t key = keys[i];
    int cx = key % P.nx;
    int cy = (key / P.nx) % P.ny;
    int cz = key / (P.nx * P.ny);
    double xi = x0[i], yi = x1[i], zi = P.dim == 3 ? x2[i] : 0.0;
    uint32_t nf = 0, nw = 0;
    unsigned long long hs = 0;
    int kz = P.dim == 3 ? 1 : 0;
    for (int dz = -kz; dz <= kz; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          int a = cx + dx, b = cy + dy, z = cz + dz;
          if (a < 0 || a >= P.nx || b < 0 || b >= P.ny || z < 0 || z >= P.nz) continue;
          uint32_t c = ((uint32_t)z * P.ny + b) * P.nx + a;
          for (uint32_t j = B.cell_begin[c]; j < B.cell_begin[c + 1]; ++j) {
            if ((int)j == i) continue;
            double d2 = dist2_exact(xi, yi, zi, x0[j], x1[j], P.dim == 3 ? x2[j] : 0.0);
            if (d2 >= P.r2max) continue;
            nf++;
            hs += splitmix64(id[j]);
          }
          if (P.nw > 0)
            for (uint32_t w = B.wall_cb[c]; w < B.wall_cb[c + 1]; ++w) {
              double d2 = dist2_exact(xi, yi, zi, wx[w], wy[w], P.dim == 3 ? wz[w] : 0.0);
              if (d2 >= P.r2max) continue;
              nw++;
              hs += splitmix64((1ull << 40) + B.wall_id[w]);
            }
        }
    uint32_t u = id[i];
    cnt_f[u] = nf;
    cnt_w[u] = nw;
    hash[u] = hs;
  }
}

__global__ void k_deinterleave(const double* __restrict__ aos, int n, int dim, double* s0,
                               double* s1, double* s2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    s0[i] = aos[(size_t)i * dim];
    s1[i] = aos[(size_t)i * dim + 1];
    if (dim == 3) s2[i] = aos[(size_t)i * dim + 2];
  }
}

__global__ void k_init_fluid(double* rho, int fill_rho, double rho0, uint32_t* id, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (fill_rho) rho[i] = rho0;
    id[i] = (uint32_t)i;
  }
}

}  // namespace

void launch_init_fluid(double* rho, int fill_rho, double rho0, uint32_t* id, int n, cudaStream_t s) {
  int blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_init_fluid<<<blocks, 256, 0, s>>>(rho, fill_rho, rho0, id, n);
}

void launch_deinterleave(const double* aos, int n, int dim, double* const soa[3], cudaStream_t s) {
  int blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  k_deinterleave<<<blocks, 256, 0, s>>>(aos, n, dim, soa[0], soa[1], soa[2]);
}

int bits_for(uint32_t ncell) {
  int b = 1;
  while (b < 32 && ((ncell - 1) >> b) != 0) ++b;
  return b;
}

int radix_passes_for(int key_bits, int radix_bits) {
  return (key_bits + radix_bits - 1) / radix_bits;
}

void launch_cell_keys(const Params& P, const LaunchCfg& L, const double* const x[3],
                      uint32_t* keys, uint32_t* vals, int n, DevScalars* sc, int gated,
                      uint32_t* digit_total, cudaStream_t s) {
  XSet xs;
  for (int k = 0; k < 3; ++k) xs.x[0][k] = xs.x[1][k] = x[k];
  int blocks = (n + L.block_stream - 1) / L.block_stream;
  if (blocks > L.blocks_stream) blocks = L.blocks_stream;
  if (blocks < 1) blocks = 1;
  k_cell_keys<<<blocks, L.block_stream, 0, s>>>(P, xs, keys, vals, n, sc, gated, digit_total,
                                                1 << L.radix_bits);
}

// variant reading the live copy x[par]
void launch_cell_keys_par(const Params& P, const LaunchCfg& L, double* const x[2][3],
                          uint32_t* keys, uint32_t* vals, int n, DevScalars* sc, int gated,
                          uint32_t* digit_total, cudaStream_t s) {
  XSet xs;
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k < 3; ++k) xs.x[p][k] = x[p][k];
  int blocks = (n + L.block_stream - 1) / L.block_stream;
  if (blocks > L.blocks_stream) blocks = L.blocks_stream;
  if (blocks < 1) blocks = 1;
  k_cell_keys<<<blocks, L.block_stream, 0, s>>>(P, xs, keys, vals, n, sc, gated, digit_total,
                                                1 << L.radix_bits);
}

static size_t hist_smem(int bins) { return (size_t)(kSortThreads / 32) * bins * sizeof(uint32_t); }
static size_t scatter_smem(int bins) {
  return ((size_t)(kSortThreads / 32) * bins + 2 * (size_t)bins + 2 * (size_t)kSortTile) *
         sizeof(uint32_t);
}

cudaError_t configure_sort_kernels() {
  cudaError_t e = cudaFuncSetAttribute(k_radix_hist<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)hist_smem(1 << kMaxRadixBits));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_radix_hist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)hist_smem(1 << kMaxRadixBits));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)scatter_smem(1 << kMaxRadixBits));
}

namespace {
int radix_sort_impl(const LaunchCfg& L, uint32_t* keys[2], uint32_t* vals[2], int n,
                    uint32_t* tile_hist, uint32_t* digit_total, const DevScalars* sc, int gated,
                    const int* n_dev, cudaStream_t s) {
  const int tiles = (n + kSortTile - 1) / kSortTile;
  int cur = 0;
  if (n <= 0) return 0;
  for (int pass = 0; pass < L.radix_passes; ++pass) {
    const int shift = pass * L.radix_bits;
    int bits = L.key_bits - shift;
    if (bits > L.radix_bits) bits = L.radix_bits;
    const uint32_t mask = (1u << bits) - 1u;
    const int bins = (int)mask + 1;
    if (L.hist_ballot)
      k_radix_hist<true><<<tiles, kSortThreads, hist_smem(bins), s>>>(
          keys[cur], n, shift, mask, tile_hist, digit_total, tiles, sc, gated, n_dev);
    else
      k_radix_hist<false><<<tiles, kSortThreads, hist_smem(bins), s>>>(
          keys[cur], n, shift, mask, tile_hist, digit_total, tiles, sc, gated, n_dev);
    k_radix_scan<<<bins, 256, 0, s>>>(tile_hist, digit_total, tiles, sc, gated, n_dev);
    k_radix_scatter<<<tiles, kSortThreads, scatter_smem(bins), s>>>(
        keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n, shift, mask, tile_hist, tiles, sc,
        gated, digit_total, n_dev);
    cur ^= 1;
  }
  return cur;
}
}  // namespace

int launch_radix_sort(const LaunchCfg& L, uint32_t* keys[2], uint32_t* vals[2], int n,
                      uint32_t* tile_hist, uint32_t* digit_total, const DevScalars* sc,
                      int gated, cudaStream_t s) {
  return radix_sort_impl(L, keys, vals, n, tile_hist, digit_total, sc, gated, nullptr, s);
}

int launch_radix_sort_dev(const LaunchCfg& L, uint32_t* keys[2], uint32_t* vals[2], int n_max,
                          uint32_t* tile_hist, uint32_t* digit_total, const int* n_dev,
                          cudaStream_t s) {
  return radix_sort_impl(L, keys, vals, n_max, tile_hist, digit_total, nullptr, 0, n_dev, s);
}

void launch_cell_offsets(const uint32_t* keys, int n, uint32_t ncell, uint32_t* cell_begin,
                         DevScalars* sc, int gated, int flip_par, cudaStream_t s) {
  int blocks = (int)((ncell + kOffsetsChunk - 1) / kOffsetsChunk);
  k_cell_offsets<<<blocks, 256, 0, s>>>(keys, n, ncell, cell_begin, sc, gated, flip_par);
}

void launch_control(const Params& P, DevScalars* sc, cudaStream_t s) {
  k_control<<<1, 1, 0, s>>>(P, sc, cudaGraphConditionalHandle{}, 0);
}

void launch_control_cond(const Params& P, DevScalars* sc, cudaGraphConditionalHandle cond,
                         cudaStream_t s) {
  k_control<<<1, 1, 0, s>>>(P, sc, cond, 1);
}

void launch_batch_control(const BatchArgs& A, int tile, int force, cudaStream_t s) {
  const int threads = ((A.ntanks + 31) / 32) * 32;
  kb_control<<<1, threads < 32 ? 32 : threads, 0, s>>>(A, tile, force);
}

void launch_batch_cell_keys(const BatchArgs& A, const WorkList* wl, int walls,
                            double* const x[2][3], uint32_t* keys, uint32_t* vals,
                            uint32_t* digit_total, int bins, int grid, int block,
                            cudaStream_t s) {
  XSet xs;
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k < 3; ++k) xs.x[p][k] = x[p][k];
  kb_cell_keys<<<grid < 1 ? 1 : grid, block, 0, s>>>(A, wl, walls, xs, keys, vals, digit_total,
                                                     bins);
}

void launch_batch_cell_offsets(const BatchArgs& A, const WorkList* wl, int walls, int grid,
                               const uint32_t* keys, uint32_t* cb, int flip_par,
                               cudaStream_t s) {
  kb_cell_offsets<<<grid < 1 ? 1 : grid, 256, 0, s>>>(A, wl, walls, keys, cb, flip_par);
}

void launch_batch_vmax(const BatchArgs& A, const DevBuffers& B, int grid, int block,
                       cudaStream_t s) {
  kb_vmax<<<grid < 1 ? 1 : grid, block, 0, s>>>(A, B);
}

void launch_vmax_reset(const Params& P, const LaunchCfg& L, const DevBuffers& B,
                       cudaStream_t s) {
  cudaMemsetAsync(&B.sc->vmax2_cur, 0, sizeof(unsigned long long), s);
  int blocks = (P.n + L.block_stream - 1) / L.block_stream;
  if (blocks > L.blocks_stream) blocks = L.blocks_stream;
  if (blocks < 1) blocks = 1;
  k_vmax<<<blocks, L.block_stream, 0, s>>>(P, B, P.n);
}

void launch_state_range(const Params& P, const LaunchCfg& L, const DevBuffers& B, uint32_t id0,
                        uint32_t m, double* buf, int field, int put, int pair_is_float,
                        cudaStream_t s) {
  int blocks = (P.n + L.block_stream - 1) / L.block_stream;
  if (blocks > L.blocks_stream) blocks = L.blocks_stream;
  if (blocks < 1) blocks = 1;
  k_state_range<<<blocks, L.block_stream, 0, s>>>(P, B, id0, m, buf, field, put, pair_is_float);
}

void launch_state_rows(const Params& P, const LaunchCfg& L, const DevBuffers& B, uint32_t id0,
                       uint32_t m, double* rows, int put, int pair_is_float, cudaStream_t s) {
  int blocks = (P.n + L.block_stream - 1) / L.block_stream;
  if (blocks > L.blocks_stream) blocks = L.blocks_stream;
  if (blocks < 1) blocks = 1;
  k_state_rows<<<blocks, L.block_stream, 0, s>>>(P, B, id0, m, rows, put, pair_is_float);
}

void launch_vmax_owned(const Params& P, const LaunchCfg& L, const DevBuffers& B, uint32_t n_own,
                       unsigned long long* out, cudaStream_t s) {
  int blocks = (P.n + L.block_stream - 1) / L.block_stream;
  if (blocks > L.blocks_stream) blocks = L.blocks_stream;
  if (blocks < 1) blocks = 1;
  k_vmax_owned<<<blocks, L.block_stream, 0, s>>>(P, B, n_own, out);
}

void launch_neighbour_stats(const Params& P, const LaunchCfg& L, const DevBuffers& B,
                            const double* wall_xyz, uint32_t* cnt_f, uint32_t* cnt_w,
                            unsigned long long* hash, cudaStream_t s) {
  int blocks = (P.n + 127) / 128;
  if (blocks < 1) blocks = 1;
  const double* wx = wall_xyz;
  const double* wy = wall_xyz ? wall_xyz + P.nw : nullptr;
  const double* wz = wall_xyz ? wall_xyz + 2 * (size_t)P.nw : nullptr;
  k_neighbour_stats<<<blocks, 128, 0, s>>>(P, B, wx, wy, wz, cnt_f, cnt_w, hash);
}

}  // namespace sphgb
