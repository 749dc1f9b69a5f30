// Internal layout of the GB300 SPH library: parameters, device scalars,
// state buffers and the launch interface shared by the translation units.
//
// Data layout in HBM (n fluid particles, storage order = sorted by cell key of
// the last rebuild):
//   state, two copies (ping-pong, `par` selects the live one; the reorder
//   after each sort gathers from one copy into the other):
//     x[3], v[3]   double SoA
//     rho          double
//     drho         T (double in FP64 mode, float in mixed mode)
//     id           uint32 user index
//   aprior[3]      T   gravity + viscous acceleration (recomputed per rebuild)
//   records, two buffers (written by one stage, read by the next neighbour loop):
//     3D  P = (x, y, z, p)   S = (vx, vy, vz, rho)      T4 / T4
//     2D  P = (x, y, vx, vy) S = (p, rho)               T4 / T2
//   with positions absolute in FP64 mode and cell-centre offsets
//   x - (lo + (c + 1/2) s) of the binned cell c in mixed mode (s = 2h
//   rounded to float).
//   mixed mode also keeps fixed-point offsets (2^28 units per cell edge) of the
//   positions at the last rebuild, for the exact density summation (int4 / int2)
//   keys (sorted cell keys), perm, cell_begin[ncell + 1]   uint32
//   wall: positions (T4 / T2, same convention), cell_begin, ids
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include <cmath>

namespace sphgb {
// Cells along one axis of a grid of edge cs over [lo, hi): ceil((hi - lo) / cs),
// at least 1.  The quotient is range-checked as a double before any cast:
// -1 when it is not a finite count of at most 2^30 cells (a tiny or zero
// edge, an infinite extent, NaN), which the callers turn into SPH_E_INVALID.
inline long long grid_cells(double lo, double hi, double cs) {
  const double r = std::ceil((hi - lo) / cs);
  if (!(r <= (double)(1ll << 30))) return -1;
  return r < 1.0 ? 1 : (long long)r;
}
}  // namespace sphgb

namespace sphgb {

constexpr int kMaxRadixBits = 11;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;  // keys per thread per tile
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kOffsetsChunk = 2048;  // cells per block of the offsets kernel

// stages of one acoustic step (same numbering as enum sph_stage)
enum {
  kStageControl = 0,
  kStageKeys,
  kStageSort,
  kStageReorder,
  kStageOffsets,
  kStageDensitySum,
  kStageViscous,
  kStageHalf1,
  kStagePressure,
  kStageDensityRelax,
  kStages
};

constexpr int kVariantNoRiemann = 1;
constexpr int kVariantBlended = 2;
constexpr int kVariantTransport = 4;  // transport-velocity correction each advection step
constexpr int kVariantMovingWall = 8;  // walls with a prescribed (sliding) velocity
// some walls translate with their velocity: binned again at every rebuild,
// moved with the fluid's half-drifts
constexpr int kVariantTranslatingWall = 16;
// some translating walls also oscillate: their acceleration enters the wall
// pressure, p_w = p_i + rho_i (x_w - x_i).(g - a_w)
constexpr int kVariantAccelWall = 32;

// error flag bits (sticky, device)
constexpr int kFlagOutOfDomain = 1;
constexpr int kFlagNonFinite = 2;
constexpr int kFlagIndex = 4;  // debug builds: an index check failed (the access was skipped)

struct Params {
  int dim;
  int n;        // fluid particles
  int nw;       // wall particles
  int nx, ny, nz;
  uint32_t ncell;
  double lo[3];
  double cs;     // cell edge = 2h
  double h;
  double r2max;  // (2h)^2, computed as 4.0 * h * h
  double rho0, c0, c0sq, mu, U_ref;
  double g[3];
  double m;       // fluid particle mass rho0 dp^dim
  double V;       // dp^dim
  double sigma0;  // lattice kernel sum
  double walpha;  // Wendland alpha_d
  double eps;     // 0.01 h viscous regulariser
  int diag;       // store acc / sigma
  int use_list;   // neighbour lists enabled
  int list_cap;   // list capacity (entries per particle)
  double skin_max;
  // method variants: kVariantNoRiemann -> the density relaxation takes the
  // average of the two states instead of the Riemann U*; kVariantBlended ->
  // blended free-surface density reinitialisation instead of the clamp;
  // kVariantTransport -> transport-velocity correction after the summation;
  // kVariantMovingWall -> the wall terms read the prescribed wall velocity;
  // kVariantTranslatingWall -> some walls move with their velocity;
  // kVariantAccelWall -> some of them oscillate (wall_omega, wall_amp)
  int variant;
  double wall_vmax;   // bound on a translating wall's speed (0 when none translates)
  double wall_omega;  // angular frequency of the walls' oscillation
  // position of this tank in the arrays of a batch (all zero for one tank):
  // first fluid slot, first wall slot, first entry of its cell offsets
  int foff, woff;
  uint32_t cell_base;
};

// Schedule scalars, resident on the device.
struct DevScalars {
  double t, tau, dt_ad, dt_ac;
  unsigned long long vmax2_cur;   // bit pattern of max |v|^2 of the current velocities
  unsigned long long vmax2_next;  // accumulated by the pressure stage
  long long n_ac, n_adv;
  int new_adv;  // this step begins an advection step
  int started;
  int par;      // live state copy
  int flags;    // sticky error bits
  // neighbour-list bookkeeping (see the list section of sph_stages.cuh)
  double skin;   // twice the largest drift budget of the current advection step
  int list_bad;  // a list overflowed its capacity in this advection step
  int pad_;
  double t0;     // start time of the current acoustic step
  double t_reb;  // time of the last rebuild (translating walls were binned then)
  // neighbour-list validity since the rebuild: some particle has left its
  // drift budget at the positions the pressure loop (and, at the rebuild, the
  // viscous loop) reads / at those the density relaxation reads
  int drift_bad_p, drift_bad_r;
  double wall_budget;  // drift budget of every wall particle (translating walls)
};

template <class T>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<double> {
  using type = double4_32a;
};
template <class T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

// Bricks of 2^kBrickLog2 cells along each axis over a one-tank grid (the
// processing order of the 3D mixed neighbour loops).
constexpr int kBrickLog2X = 2, kBrickLog2Y = 2, kBrickLog2Z = 2;
inline __host__ __device__ uint32_t brick_count(const Params& P) {
  const int bx = (P.nx + (1 << kBrickLog2X) - 1) >> kBrickLog2X;
  const int by = (P.ny + (1 << kBrickLog2Y) - 1) >> kBrickLog2Y;
  const int bz = (P.nz + (1 << kBrickLog2Z) - 1) >> kBrickLog2Z;
  return (uint32_t)(bx * by * bz);
}

// Raw device pointers of one context (all owned by the context).
struct DevBuffers {
  double* x[2][3];
  double* v[2][3];
  double* rho[2];
  void* drho[2];  // T
  uint32_t* id[2];
  void* aprior[3];  // T
  void* acc[3];     // T, diagnostics
  void* sigma;      // T, diagnostics
  double* sigma64;  // kernel sum of the last summation (transport correction's support test)
  // loop records.  3D: 8 T per slot, the position record (T 0-3) and the
  // state record (T 4-7) side by side; rec_s unused.  2D: the position
  // records (4 T per slot) in rec, the state records (2 T) in rec_s.
  void* rec[2];
  void* rec_s[2];
  void* recI;       // mixed mode: int4 (3D) / int2 (2D) fixed-point offsets at the rebuild
  uint32_t* nl;     // neighbour lists: entry k of particle i at ((i/32) cap + k) 32 + i%32
  uint32_t* nl_cnt; // list length per particle
  void* xreb[3];  // position of every slot at the last rebuild, record frame (T)
  float* bud;     // drift budget of every slot since the last rebuild
  // what the list build reads of every slot: Vec4<T> (x, y, z, b), its
  // record-frame position (2D: z = 0) and drift budget
  void* brec;
  // processing order of the one-tank 3D mixed neighbour loops: the 32-slot
  // groups sorted by brick of 4 x 4 x 4 cells and split into `parts` equal
  // runs, each taken group by group by the warps of one multiprocessor (a
  // warp that finds its run done takes groups from the others)
  uint32_t* units;        // ceil(n / 32) group indices, brick order
  uint32_t* unit_brick;   // brick of every group at the last rebuild
  uint32_t* brick_start;  // nbrick + 1: counts, then starts
  uint32_t* brick_fill;   // nbrick
  uint32_t* unit_ctr;     // 5 x parts claim counters: pressure, relaxation (zeroed by
                          // the first half-step), list build, density summation,
                          // viscous force (zeroed with the brick order)
  int parts;
  uint32_t* keys[2];  // sort ping-pong; keys[sorted_buf] holds the sorted keys
  uint32_t* vals[2];
  int sorted_buf;
  // binned cell key of every storage slot (the cell of the last rebuild, in
  // its tank's grid): keys[sorted_buf] for one tank, a separate array in a batch
  const uint32_t* binned;
  // mixed path: cell-centre coordinates per axis (nx | ny | nz doubles) of the
  // record frame; null where the kernels compute them (FP64 path, batches)
  const double* ctab;
  uint32_t* tile_hist;  // bins x tiles
  uint32_t* digit_total;
  uint32_t* cell_begin;  // ncell + 1
  // wall
  void* wallP;  // T4 / T2
  uint32_t* wall_cb;
  uint32_t* wall_id;
  double* wall_xyz;  // sorted wall positions, double SoA (3 nw)
  void* wallI;       // mixed mode: wall fixed-point offsets (int4 / int2)
  void* wall_vel;    // prescribed wall velocity (T4 / T2, sorted), null when every wall rests
  // walls as given (user order, double SoA x | y | z of nw each): positions,
  // velocities (null: all at rest)
  const double* wall_x0;
  const double* wall_v0;
  // translating walls: flags (user order; null: none translates), positions
  // placed at the binning time (user order SoA) and the wall sort's own
  // ping-pong and histogram buffers
  const uint8_t* wall_moves;
  const double* wall_amp;  // oscillation amplitudes (user order SoA), null: none
  void* wall_acc;          // wall accelerations (T4 / T2, sorted), null: none
  double* wall_io;
  uint32_t* wall_key;  // binned cell key of each sorted wall
  uint32_t* wkeys[2];
  uint32_t* wvals[2];
  uint32_t* wtile_hist;
  DevScalars* sc;
  int* dbg_flags;  // where debug-build index checks record kFlagIndex
  double* io;  // staging, n * dim doubles (also wall staging)
  uint32_t* u32_io;
  unsigned long long* u64_io;
};

// Debug builds (-DSPH_DEBUG): index checks that record kFlagIndex and skip
// the access instead of trapping, the stand-in for a memory checker; release
// builds compile them away.  SPH_DBG_IN(B, i, lo, hi) is lo <= i < hi.
#ifdef SPH_DEBUG
__device__ __forceinline__ bool dbg_in(const DevBuffers& B, long long i, long long lo,
                                       long long hi) {
  if (i >= lo && i < hi) return true;
  if (B.dbg_flags) atomicOr(B.dbg_flags, kFlagIndex);
  return false;
}
#define SPH_DBG_IN(B, i, lo, hi) \
  ::sphgb::dbg_in((B), (long long)(i), (long long)(lo), (long long)(hi))
#else
#define SPH_DBG_IN(B, i, lo, hi) true
#endif

struct LaunchCfg {
  int sms;           // multiprocessors
  int block_loop;    // threads per block of the neighbour loops
  int blocks_loop;   // persistent grid of the neighbour loops
  int block_stream;  // threads per block of the streaming kernels
  int blocks_stream;
  int radix_bits;
  int radix_passes;
  int key_bits;
  int tiles;  // radix tiles
  // 1: the sort histograms group equal digits by ballots, not __match_any_sync
  // (faster for keys in random order, slower for nearly sorted ones)
  int hist_ballot = 0;
};

// ---------------------------------------------------------------------------
// Batches of independent tanks.  Tank t owns the fluid slots
// [foff, foff + n), the wall slots [woff, woff + nw) and the cell offsets
// [cell_base, cell_base + ncell] of the shared arrays (its Params), and its
// own schedule (DevScalars).  Every batched stage is one persistent launch
// whose blocks walk a work list: the tiles of `tile` slots of the listed
// tanks, or (cell offsets) their chunks of kOffsetsChunk cells.  A tank's
// cell key in the batch-wide sort is cell_base + its cell index, so one
// stable sort keeps every tank's particles inside its own range.
constexpr int kMaxTanks = 1024;

struct WorkList {
  int count;   // listed tanks
  int tiles;   // total tiles
  int chunks;  // total offset chunks
  int m;       // total slots of the listed tanks (length of the compacted sort)
  int tile;    // slots per tile
  int pad_[3];
  int tank[kMaxTanks];
  int tile_prefix[kMaxTanks + 1];
  int chunk_prefix[kMaxTanks + 1];
  int cbase[kMaxTanks];  // first compacted sort slot of each listed tank
};

// Device-side view of a batch, passed by value to the batched kernels.
struct BatchArgs {
  const Params* tP;    // per tank
  const void* tK;      // per tank KC<T> of the pair type
  DevScalars* tsc;     // per tank
  WorkList* wl_all;    // every tank (static)
  WorkList* wl_adv;    // tanks that begin an advection step (schedule kernel)
  WorkList* wl_wall;   // every tank, wall tiles (static)
  uint32_t* bkey;      // binned cell key of every fluid slot
  int ntanks;
  int n_total, nw_total;
  int tiles_max;       // tiles of wl_all: bound of every fluid list (grid sizing)
  int chunks_max;      // offset chunks of every tank
  const double* ctab;  // mixed path: every tank's cell-centre table (or null)
  const int* ctab_off; // first entry of each tank's table
};

struct BatchStageArgs {
  BatchArgs A;
  DevBuffers B;  // shared arrays; B.sc unused, B.binned = A.bkey
  LaunchCfg L;
  int dim;
  int variants;  // union of the tanks' method variants (which stages to launch)
};

// batched schedule kernel: per-tank dual-criteria schedule, then the list of
// tanks that begin an advection step (force: every tank with fluid, schedule
// untouched -- the initial sort)
void launch_batch_control(const BatchArgs& A, int tile, int force, cudaStream_t s);
// batched cell keys of the listed tanks into compacted sort slots (walls: from
// the staging SoA x[0]; fluid: from the live copy x[par] of each tank); block 0
// clears the digit totals of the sort
void launch_batch_cell_keys(const BatchArgs& A, const WorkList* wl, int walls,
                            double* const x[2][3], uint32_t* keys, uint32_t* vals,
                            uint32_t* digit_total, int bins, int grid, int block,
                            cudaStream_t s);
// batched CSR offsets of the listed tanks from the compacted sorted keys
// (256 threads per block)
void launch_batch_cell_offsets(const BatchArgs& A, const WorkList* wl, int walls, int grid,
                               const uint32_t* keys, uint32_t* cb, int flip_par,
                               cudaStream_t s);
// fresh max |v|^2 per tank (live copy) into vmax2_cur (walks wl_all)
void launch_batch_vmax(const BatchArgs& A, const DevBuffers& B, int grid, int block,
                       cudaStream_t s);

void enqueue_batch_step_fp64(const BatchStageArgs& a, cudaStream_t s, cudaEvent_t* ev = nullptr);
void enqueue_batch_step_mixed(const BatchStageArgs& a, cudaStream_t s, cudaEvent_t* ev = nullptr);
void enqueue_batch_initial_sort_fp64(const BatchStageArgs& a, cudaStream_t s);
void enqueue_batch_initial_sort_mixed(const BatchStageArgs& a, cudaStream_t s);
// walls of every tank from the staging SoA B.io ([x | y | z], nw_total each);
// sort scratch in a.B.keys / vals / tile_hist
void enqueue_batch_wall_setup_fp64(const BatchStageArgs& a, cudaStream_t s);
void enqueue_batch_wall_setup_mixed(const BatchStageArgs& a, cudaStream_t s);

// --- launch interface implemented per precision (sph_fp64.cu / sph_mixed.cu)
struct StageArgs {
  Params P;
  DevBuffers B;
  LaunchCfg L;
};

// Queue one acoustic step (device-decided rebuild included).  When ev is
// given (kStages + 1 events), ev[k] is recorded before stage k and
// ev[kStages] after the last stage.
void enqueue_step_fp64(const StageArgs& a, cudaStream_t s, cudaEvent_t* ev = nullptr);
void enqueue_step_mixed(const StageArgs& a, cudaStream_t s, cudaEvent_t* ev = nullptr);
// The two parts of a step for a graph with a conditional node: the stages of a
// step that begins an advection step (rebuild, lists, density summation,
// viscous force; launched ungated) and the acoustic stages of every step.
void enqueue_advection_fp64(const StageArgs& a, cudaStream_t s);
void enqueue_advection_mixed(const StageArgs& a, cudaStream_t s);
void enqueue_acoustic_fp64(const StageArgs& a, cudaStream_t s);
void enqueue_acoustic_mixed(const StageArgs& a, cudaStream_t s);
// rho = rho0 where fill_rho, id = 0..n-1
void launch_init_fluid(double* rho, int fill_rho, double rho0, uint32_t* id, int n, cudaStream_t s);
// AoS (n x dim) -> SoA copy on the device
void launch_deinterleave(const double* aos, int n, int dim, double* const soa[3], cudaStream_t s);
// Initial binning / sort after set_particles (forces a rebuild of the cell
// list and builds the records without changing the schedule).
void enqueue_initial_sort_fp64(const StageArgs& a, cudaStream_t s);
// the cell-centre table of the mixed path's record frame (nx + ny + nz doubles)
void launch_centre_table(const Params& P, double* tab, cudaStream_t s);
void enqueue_initial_sort_mixed(const StageArgs& a, cudaStream_t s);
// Wall setup: keys, sort, wall records and wall cell offsets from the
// staging buffer io (double SoA [x | y | z], nw each, user order).  The sort
// runs in the keys / vals / tile_hist buffers of `a.B`, which the caller sets
// to scratch of its own so that the fluid's sorted keys survive.
void enqueue_wall_setup_fp64(const StageArgs& a, cudaStream_t s);
void enqueue_wall_setup_mixed(const StageArgs& a, cudaStream_t s);
// Walls binned again: positions x0 + t v0 for the translating walls, x0 for
// the others, at the current time (sc->t), or with at_rebuild at the time of
// the last rebuild (sc->t_reb) and then moved on to the current time (a
// restored state); the sort runs in the wall buffers of `a.B` (wall_io,
// wkeys, wvals, wtile_hist), then the gather and the wall offsets.
void enqueue_wall_rebin_fp64(const StageArgs& a, cudaStream_t s, int at_rebuild);
void enqueue_wall_rebin_mixed(const StageArgs& a, cudaStream_t s, int at_rebuild);
// Neighbour lists of a restored state, built from its current positions with
// its stored skin (the loops then give the sums of the uninterrupted run).
void enqueue_restore_lists_fp64(const StageArgs& a, cudaStream_t s);
void enqueue_restore_lists_mixed(const StageArgs& a, cudaStream_t s);
// Brick processing order of the 3D mixed loops from the binned keys as they
// stand (a restored state; the rebuild makes it otherwise).
void enqueue_units_mixed(const StageArgs& a, cudaStream_t s);

// --- neighbour search (sph_nsearch.cu), precision independent
// keys from positions x[par] (or an explicit coordinate set), vals = iota
void launch_cell_keys(const Params& P, const LaunchCfg& L, const double* const x[3],
                      uint32_t* keys, uint32_t* vals, int n, DevScalars* sc, int gated,
                      uint32_t* digit_total, cudaStream_t s);
void launch_cell_keys_par(const Params& P, const LaunchCfg& L, double* const x[2][3],
                          uint32_t* keys, uint32_t* vals, int n, DevScalars* sc, int gated,
                          uint32_t* digit_total, cudaStream_t s);
// dynamic shared memory limits of the sort kernels (call once per device)
cudaError_t configure_sort_kernels();
// stable LSD radix sort of (keys[0], vals[0]) with ping-pong into [1];
// returns the buffer index that holds the result
int launch_radix_sort(const LaunchCfg& L, uint32_t* keys[2], uint32_t* vals[2], int n,
                      uint32_t* tile_hist, uint32_t* digit_total, const DevScalars* sc,
                      int gated, cudaStream_t s);
// the same sort over the first *n_dev entries (a count decided on the device,
// at most n_max)
int launch_radix_sort_dev(const LaunchCfg& L, uint32_t* keys[2], uint32_t* vals[2], int n_max,
                          uint32_t* tile_hist, uint32_t* digit_total, const int* n_dev,
                          cudaStream_t s);
// CSR offsets from sorted keys; if flip_par, thread 0 flips sc->par afterwards
void launch_cell_offsets(const uint32_t* keys, int n, uint32_t ncell, uint32_t* cell_begin,
                         DevScalars* sc, int gated, int flip_par, cudaStream_t s);
// schedule control kernel (one thread)
void launch_control(const Params& P, DevScalars* sc, cudaStream_t s);
// the same, also setting the graph conditional `cond` to "this step begins an
// advection step"
void launch_control_cond(const Params& P, DevScalars* sc, cudaGraphConditionalHandle cond,
                         cudaStream_t s);
// fresh max |v|^2 of x[par] copy into vmax2_cur
void launch_vmax_reset(const Params& P, const LaunchCfg& L, const DevBuffers& B,
                       cudaStream_t s);
// debug neighbour statistics (double positions of the live copy)
// State of the particles with user ids [id0, id0 + m) gathered into (put = 0)
// or scattered from (put = 1) the device array buf in user-id order; field 0
// position, 1 velocity, 2 density, 3 density rate, 4 prior acceleration.
void launch_state_range(const Params& P, const LaunchCfg& L, const DevBuffers& B, uint32_t id0,
                        uint32_t m, double* buf, int field, int put, int pair_is_float,
                        cudaStream_t s);
// the same as packed rows (3 dim + 2 doubles per particle: position,
// velocity, density, density rate, prior acceleration), device memory
void launch_state_rows(const Params& P, const LaunchCfg& L, const DevBuffers& B, uint32_t id0,
                       uint32_t m, double* rows, int put, int pair_is_float, cudaStream_t s);
// max |v|^2 of the particles with user ids below n_own, atomically maxed into *out
void launch_vmax_owned(const Params& P, const LaunchCfg& L, const DevBuffers& B, uint32_t n_own,
                       unsigned long long* out, cudaStream_t s);
void launch_neighbour_stats(const Params& P, const LaunchCfg& L, const DevBuffers& B,
                            const double* wall_xyz, uint32_t* cnt_f, uint32_t* cnt_w,
                            unsigned long long* hash, cudaStream_t s);

// Work-list walkers: f(list position, first slot of the tile within the tank,
// tile length) for every tile of the list, tiles dealt round-robin to blocks;
// the tank of a tile is found by binary search in the prefix of tile counts
// (tanks without tiles are skipped by taking the last position <= w).
__device__ __forceinline__ int wl_find(const int* __restrict__ prefix, int count, int w) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}
template <class F>
__device__ __forceinline__ void for_each_tile(const WorkList* __restrict__ wl, F&& f) {
  const int total = wl->tiles, cnt = wl->count, tile = wl->tile;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int a = wl_find(wl->tile_prefix, cnt, w);
    f(a, (w - wl->tile_prefix[a]) * tile, tile);
  }
}
template <class F>
__device__ __forceinline__ void for_each_chunk(const WorkList* __restrict__ wl, F&& f) {
  const int total = wl->chunks, cnt = wl->count;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    const int a = wl_find(wl->chunk_prefix, cnt, w);
    f(a, w - wl->chunk_prefix[a]);
  }
}

int radix_passes_for(int key_bits, int radix_bits);
int bits_for(uint32_t ncell);

// Cell index along one axis: floor(fl((x - lo) / cs)) with a correctly rounded
// subtraction and division, clamped into [0, nc - 1] (oob set when clamped or
// not finite).  The quotient is first formed in float; when it lies farther
// from the nearest integer than its worst-case error (three float roundings,
// < 2e-7 relative), the double quotient has the same floor and the division
// is skipped.  Only coordinates within that distance of a cell face take the
// double division, so the result always equals the plain double formula.
// On that path fq is an integer below 2^20 (a larger quotient has no
// fractional bits in float and takes the double path), so the clamp and the
// conversion run in float and int, off the FP64 pipe.
__device__ __forceinline__ int cell_coord_fast(double x, double lo, double cs, float inv_cs,
                                               int nc, int& oob) {
  const double d = __dsub_rn(x, lo);
  const float qf = __fmul_rn((float)d, inv_cs);
  const float fq = floorf(qf);
  const float dist = fminf(qf - fq, fq + 1.0f - qf);
  if (dist > 1e-6f * fabsf(qf) + 4e-6f) {
    if (!(fq >= 0.0f)) {
      oob = 1;
      return 0;
    }
    const int c = (int)fq;
    if (c >= nc) {
      oob = 1;
      return nc - 1;
    }
    return c;
  }
  const double f = floor(__ddiv_rn(d, cs));
  if (!(f >= 0.0)) {
    oob = 1;
    return 0;
  }
  if (f >= (double)nc) {
    oob = 1;
    return nc - 1;
  }
  return (int)f;
}

}  // namespace sphgb
