/*
 * sph.h - C ABI of the GB300 weakly-compressible SPH hot path (libsph.so).
 *
 * What the library computes.  Hu & Guarnieri, "Towards heterogeneous
 * parallelism for SPHinXsys", describe a three-layer pattern: an outer layer
 * that defines the problem (global parameters, particles generated from the
 * geometry), a kernel-shell layer that hands per-particle arrays and scalars to
 * the computing kernels, and the kernels themselves (section "Implementing
 * SYCL kernels in SPHinXsys").  The calls below are that outer layer:
 * sph_create takes the domain, the particle spacing, the smoothing length,
 * the material and gravity; sph_set_particles hands over the particles;
 * sph_step advances; sph_get_fields reads results back.  The device work is
 * the paper's cell-linked list, particle sorting and direct search (section
 * "Cell linked-list, direct search and sorting") driving the weakly
 * compressible SPH interactions: Wendland C2 kernel, density summation,
 * viscous force, Riemann-based pressure and density relaxation, wall
 * particles (at rest or sliding) with a mirrored Riemann state, and the dual
 * advection / acoustic time-step criteria.
 *
 * Conventions (all entry points):
 *  - Every call returns an sph_status (0 = SPH_OK) unless stated otherwise.
 *  - Host arrays are read or written synchronously during the call; the
 *    caller keeps ownership.  Vector fields are particle-major, n * dim
 *    doubles (x0, y0[, z0], x1, ...), in USER order: the order given to
 *    sph_set_particles.
 *  - Device state belongs to the context.  It is allocated through the
 *    caller's allocator (or cudaMalloc when none is given) on the
 *    context's stream, and freed by sph_destroy.
 *  - Work is queued on the caller's CUDA stream (NULL = legacy default
 *    stream).  sph_step returns once the work is queued; device-side errors
 *    (particle outside the domain, non-finite state) are sticky and reported
 *    by the next call that synchronises (sph_synchronize, sph_get_fields,
 *    sph_get_scalars, sph_debug_*).
 *  - There is no CPU path: without a usable CUDA device the calls fail with
 *    SPH_E_CUDA.
 *  - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sph_ctx sph_ctx;

/* Axis-aligned box covered by the cell grid.  Cells have edge 2h (the cut-off
 * radius); the grid has ceil((hi - lo) / 2h) cells per axis.  Components
 * beyond dim are ignored.  Particles must stay inside [lo, hi). */
typedef struct {
  int dim;       /* 2 or 3 */
  double lo[3];
  double hi[3];
} sph_domain;

/* Weakly-compressible fluid: p = c0^2 (rho - rho0). */
typedef struct {
  double rho0;   /* reference density (> 0)                            */
  double c0;     /* artificial sound speed (> 0)                        */
  double mu;     /* dynamic viscosity (>= 0)                            */
  double U_ref;  /* reference speed of the advection criterion (> 0)   */
} sph_material;

/* Device memory provider.  alloc returns device memory of at least `bytes`
 * bytes usable on `stream`, aligned to 256 bytes as cudaMalloc's blocks are
 * (the kernels read some arrays with 16- and 32-byte vector loads).  NULL on
 * failure: the call then returns SPH_E_OOM; a block that is not so aligned
 * is handed back to free and counts as a failure.  free releases a block
 * obtained from alloc. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* user);
  void (*free)(void* ptr, size_t bytes, void* stream, void* user);
  void* user;
} sph_allocator;

enum sph_precision {
  SPH_FP64 = 0,  /* every stage in double precision                                    */
  SPH_MIXED = 1  /* pair interactions in float with float sums; positions, cell keys,
                    velocity and density state in double                               */
};

enum sph_status {
  SPH_OK = 0,
  SPH_E_INVALID = 1,        /* bad argument, or call out of order                     */
  SPH_E_OOM = 2,            /* allocation failed                                       */
  SPH_E_CUDA = 3,           /* CUDA runtime error (see sph_last_error)                 */
  SPH_E_OUT_OF_DOMAIN = 4,  /* a particle left the box: it was clamped into the edge cell */
  SPH_E_NONFINITE = 5,      /* a velocity or density became NaN or infinite            */
  SPH_E_TIMEOUT = 6,        /* sph_synchronize gave up waiting                         */
  SPH_E_STATE = 7,          /* no fluid particles set yet                              */
  SPH_E_INDEX = 8           /* debug build only: an index check failed (access skipped) */
};

enum sph_kind { SPH_FLUID = 0, SPH_WALL = 1 };

/* Field bits for sph_get_fields; fields are written one after another in
 * increasing bit order, each n values (scalars) or n * dim values (vectors). */
enum sph_field {
  SPH_F_POS = 1u << 0,    /* position (vector)                                      */
  SPH_F_VEL = 1u << 1,    /* velocity (vector)                                      */
  SPH_F_RHO = 1u << 2,    /* density                                                */
  SPH_F_P = 1u << 3,      /* pressure of the last first half-step                   */
  SPH_F_DRHO = 1u << 4,   /* density rate of the last density relaxation            */
  SPH_F_ACC = 1u << 5,    /* pressure acceleration of the last step (vector; needs
                             SPH_OPT_RECORD_DIAGNOSTICS, else zeros)                 */
  SPH_F_APRIOR = 1u << 6, /* gravity + viscous acceleration (vector)                */
  SPH_F_SIGMA = 1u << 7   /* kernel sum of the last density summation (needs
                             SPH_OPT_RECORD_DIAGNOSTICS, else zeros)                 */
};

enum sph_option {
  SPH_OPT_RECORD_DIAGNOSTICS = 1, /* 0/1: also store SPH_F_ACC and SPH_F_SIGMA        */
  SPH_OPT_USE_GRAPH = 2,          /* 0/1 (default 1): replay each step as a CUDA graph */
  SPH_OPT_BLOCK = 3,              /* threads per block of the neighbour loops: 64..256,
                                     multiple of 32 (default 128)                      */
  SPH_OPT_RADIX_BITS = 4,         /* digit width of the radix sort: 4..11 (default 8)  */
  SPH_OPT_NEIGHBOUR_LIST = 5,     /* 0/1 (default 1): the neighbour loops of an
                                     advection step walk per-particle neighbour lists
                                     built at its rebuild (candidates within 2h plus
                                     both particles' drift budgets) instead of the
                                     cells while every particle stays within its
                                     budget; results are identical either way          */
  SPH_OPT_DENSITY_RIEMANN = 6,    /* 1 (default): the density relaxation uses the
                                     Riemann interface velocity U*; 0: the plain average
                                     (U_L + U_R)/2, the dissipation-free variant, which is
                                     the textbook SPH continuity equation                */
  SPH_OPT_REINIT_BLENDED = 7,     /* 0 (default): the density summation reinitialises
                                     rho = rho0 max(sigma/sigma0, 1); 1: the blended
                                     free-surface form rho_sum + max(0, rho_prev - rho_sum)
                                     rho0 / rho_prev, rho_sum = rho0 sigma / sigma0      */
  SPH_OPT_TRANSPORT_CORRECTION = 8 /* 0 (default) / 1: transport-velocity (particle
                                     shifting) correction once per advection step, after
                                     the density summation: particles with sigma >= 0.95
                                     sigma0 move by -0.2 h^2 sum_j V_j grad_i W_ij     */
};

/* Creates a context.
 *   domain   box of the cell grid (see sph_domain)
 *   dp       initial particle spacing: fluid mass is rho0 dp^dim
 *   h        smoothing length; cut-off radius 2h, cell edge 2h
 *   mat      material (see sph_material)
 *   gravity  body acceleration, dim components used
 *   precision  SPH_FP64 or SPH_MIXED
 *   alloc    device allocator, or NULL for cudaMalloc / cudaFree
 *   stream   cudaStream_t for all work, or NULL
 *   out      receives the context
 * Fails with SPH_E_INVALID for dim not 2/3, non-positive dp/h/rho0/c0/U_ref,
 * negative mu, an empty box, or more than 2^32 - 2 cells. */
int sph_create(const sph_domain* domain, double dp, double h, const sph_material* mat,
               const double gravity[3], int precision, const sph_allocator* alloc,
               void* stream, sph_ctx** out);

/* Sets the particles of one kind (host arrays, n * dim positions).
 *   SPH_FLUID: vel (n * dim) and rho (n) may be NULL (rest, rho0).  Resets
 *     time and step counters, the carried density rate and the schedule; the
 *     particles are binned and sorted once.  User order is the given order.
 *   SPH_WALL: wall particles, which keep their positions; sorted once.  vel
 *     is NULL (walls at rest) or the prescribed velocity of each wall
 *     particle (n * dim): a wall sliding along itself (a lid, a belt, a
 *     Couette plate), whose lattice is unchanged by the motion.  The velocity
 *     enters the mirrored wall state v_R = 2 v_w - v_i of the pressure and
 *     density relaxation and the viscous force, which takes v_i - v_R =
 *     2 (v_i - v_w) for a wall neighbour; the wall pressure extrapolation is
 *     unchanged (no wall acceleration).  rho must be NULL.
 * n may be 0 and must be below 2^26.  Fails with SPH_E_INVALID on a NULL pos
 * with n > 0, on too many particles, on a wall density or on a non-finite
 * wall velocity. */
int sph_set_particles(sph_ctx* ctx, int kind, size_t n, const double* pos, const double* vel,
                      const double* rho);

/* Checkpoint / resume.  A checkpoint holds the schedule state (time, step
 * counters, advection-step clock, time steps, velocity maximum, list bounds,
 * error flags) and every fluid particle's live state in storage order:
 * position, velocity, density (double), carried density rate and prior
 * acceleration (the precision's pair type), user id and binned cell key.
 * Restored into a context with the same setup (sph_create arguments, wall
 * particles and their velocities, wall translation, method options), the
 * run continues exactly as it would have: the same bits in either precision.
 * Walls are not stored; translating walls are placed from the stored times.
 * The neighbour lists are built anew from the stored positions with the
 * stored skin; they accept the same pairs in the same order, so the sums are
 * those of the uninterrupted run.
 *
 * sph_checkpoint_bytes: size of a checkpoint of the current state (0 without
 *   fluid particles).  No synchronisation.
 * sph_checkpoint_save: writes it into buf (host, at least that many bytes);
 *   synchronises; returns the sticky device error, if any, after writing.
 *   SPH_E_STATE without fluid particles, SPH_E_INVALID for a missing or
 *   short buffer.
 * sph_checkpoint_load: replaces the fluid particles and the schedule state by
 *   the checkpoint in buf (bytes long).  SPH_E_INVALID for a buffer that is
 *   not a checkpoint of this library version, is too short, or belongs to a
 *   different setup (domain, spacing, material, gravity, precision, wall
 *   count, translation or method options). */
size_t sph_checkpoint_bytes(const sph_ctx* ctx);
int sph_checkpoint_save(sph_ctx* ctx, void* buf, size_t bytes);
int sph_checkpoint_load(sph_ctx* ctx, const void* buf, size_t bytes);

/* Makes walls translate: moves (nw bytes, user order of the last SPH_WALL
 * set) marks the wall particles that move with their prescribed velocity,
 * x_w(t) = x_w(0) + v_w t, t the simulation time and x_w(0) the position
 * given to sph_set_particles; the others keep their positions (at rest or
 * sliding).  Translating walls are binned again at every rebuild (at the
 * step's start time) and follow the fluid's half-drifts: at t + dt/2 for the
 * pressure relaxation, at t + dt for the density relaxation.  The neighbour
 * lists stay exact: their bound also covers the walls' drift since the
 * rebuild.  NULL (or all zero) clears.  The walls are binned again at once,
 * at the current time.  A new SPH_WALL set clears the translation.  A wall
 * that leaves the box is clamped and flagged like a fluid particle.
 * Single tanks only (batches have no translating walls).  SPH_E_OOM when the
 * wall buffers cannot be allocated. */
int sph_set_wall_translation(sph_ctx* ctx, const uint8_t* moves);

/* Translating walls that may also oscillate: wall u with moves[u] != 0
 * follows x_w(t) = x_w(0) + v t + A sin(omega t), A = amplitude[u * dim ..]
 * (host, nw * dim doubles, user order; NULL = no oscillation), v its given
 * velocity (zero for walls given none).  Its velocity is then
 * v + A omega cos(omega t) and its acceleration a_w = -A omega^2
 * sin(omega t), which enters the mirrored wall pressure
 * p_w = p_i + rho_i (x_w - x_i).(g - a_w).  sph_set_wall_translation(ctx,
 * moves) is this call with no amplitude.  The neighbour lists' drift bound
 * takes |v| + |A| |omega| as the wall speed.  SPH_E_INVALID for a non-finite
 * omega or amplitude; otherwise as sph_set_wall_translation. */
int sph_set_wall_motion(sph_ctx* ctx, const uint8_t* moves, double omega,
                        const double* amplitude);

/* Queues n acoustic steps of the dual-criteria schedule.  Each step: when the
 * elapsed time of the current advection step has reached its length (or on
 * the first step), a new advection step begins (length 0.25 h / max(U_ref,
 * Vmax); cell keys, stable radix sort, reorder, cell offsets, density
 * summation, viscous force); then the acoustic step of length
 * 0.6 h / (c0 + Vmax): density and position half-updates, Riemann pressure
 * relaxation and velocity kick, position half-update and Riemann density
 * relaxation.  The schedule is decided on the device.  Returns SPH_E_STATE
 * before fluid particles are set, SPH_E_INVALID for n < 0. */
int sph_step(sph_ctx* ctx, int n);

/* Waits for queued work and copies the fields selected by `mask` (sph_field
 * bits) to the host buffer `out`, in user order.  Returns a sticky device
 * error if one was raised. */
int sph_get_fields(sph_ctx* ctx, unsigned mask, double* out);

/* Waits and reads the schedule scalars; any pointer may be NULL. */
int sph_get_scalars(sph_ctx* ctx, double* t, double* dt_ad, double* dt_ac, long* n_ac,
                    long* n_adv);

/* Number of fluid / wall particles and cells (no synchronisation). */
size_t sph_count(const sph_ctx* ctx, int kind);
size_t sph_cell_count(const sph_ctx* ctx);

/* Sorted neighbour structure of the last rebuild (storage order), for parity
 * checks: keys[n] cell key of each storage slot, perm[n] pre-sort slot of
 * each storage slot, ids[n] user index of each storage slot,
 * cell_begin[ncell + 1] CSR offsets.  Any pointer may be NULL. */
int sph_debug_neighbour_state(sph_ctx* ctx, uint32_t* keys, uint32_t* perm, uint32_t* ids,
                              uint32_t* cell_begin);

/* Per fluid particle (user order), with the current positions and the cell
 * list of the last rebuild: accepted fluid neighbours (r < 2h, self
 * excluded), accepted wall particles, and an order-free fingerprint (sum of
 * SplitMix64 of the neighbours' user ids, wall ids offset by 2^40).
 * Positions are compared in double precision in both precision modes. */
int sph_debug_neighbour_stats(sph_ctx* ctx, uint32_t* cnt_fluid, uint32_t* cnt_wall,
                              uint64_t* hash);

/* Length of every fluid particle's neighbour list (storage order, n entries)
 * as built at the last rebuild: the fluid and wall candidates closer than 2h
 * plus both particles' drift budgets.  All 0 when lists are off. */
int sph_debug_list_lengths(sph_ctx* ctx, uint32_t* lengths);

/* Stages of one acoustic step, in launch order (sph_profile_stages). */
enum sph_stage {
  SPH_STAGE_CONTROL = 0,        /* schedule scalars (one thread)                   */
  SPH_STAGE_KEYS = 1,           /* cell keys from positions                        */
  SPH_STAGE_SORT = 2,           /* radix sort, all passes                          */
  SPH_STAGE_REORDER = 3,        /* gather of the state into sorted order + records */
  SPH_STAGE_OFFSETS = 4,        /* CSR cell offsets                                */
  SPH_STAGE_DENSITY_SUM = 5,    /* density summation                               */
  SPH_STAGE_VISCOUS = 6,        /* viscous force                                   */
  SPH_STAGE_HALF1 = 7,          /* first half-step                                 */
  SPH_STAGE_PRESSURE = 8,       /* pressure relaxation + kick + drift              */
  SPH_STAGE_DENSITY_RELAX = 9,  /* density relaxation                              */
  SPH_STAGE_COUNT = 10
};

/* Runs n acoustic steps launched stage by stage (no graph) with CUDA events
 * around every stage on the context's stream, and adds each stage's device
 * time in milliseconds to ms[stage] (SPH_STAGE_COUNT entries).  *rebuilds
 * receives how many of the n steps began an advection step (the stages KEYS
 * to VISCOUS do work only on those steps).  The state advances exactly as
 * with sph_step. */
int sph_profile_stages(sph_ctx* ctx, int n, double* ms, long* rebuilds);

/* Kernel launches of an acoustic step that begins an advection step (the
 * rebuild stages included).  A step inside an advection step launches 4 of
 * them (schedule, first half-step, pressure relaxation, density relaxation):
 * the step's CUDA graph holds the rest in a conditional node that the
 * schedule kernel opens or skips on the device. */
long sph_kernels_per_step(const sph_ctx* ctx);

/* ---- Standalone neighbour search (the paper's cell-linked list build and one
 * direct-search density pass, section "Cell linked-list, direct search and
 * sorting"), for measuring the neighbour search on its own. ---------------- */
typedef struct sph_nsearch sph_nsearch;

/* Creates a neighbour search on the grid of `domain` with cells of edge 2h.
 * pos_precision: SPH_FP64 for double positions, SPH_MIXED for float
 * positions.  Device memory comes from `alloc` (or cudaMalloc); work is queued
 * on `stream`.  SPH_E_INVALID on bad arguments. */
int sph_nsearch_create(const sph_domain* domain, double h, int pos_precision,
                       const sph_allocator* alloc, void* stream, sph_nsearch** out);

/* Runs, for n particles given as device SoA coordinate arrays x, y, z (float
 * or double as created; z ignored in 2D): cell keys, the stable radix sort,
 * the reorder of the positions, the CSR cell offsets, and one density pass
 * sigma_i = sum_{r_ij < 2h} W(r_ij) (self included) in the position type.
 * The coordinate arrays stay the caller's; they are read by work queued on the
 * object's stream after the caller's stream, so they must stay valid until
 * that work is done.  Positions outside the domain are clamped into the edge
 * cell.  stage_ms, if not NULL, receives the device time of the five stages
 * (and the call then waits for them).  Buffers grow as needed.  Returns
 * SPH_E_INVALID for n = 0, n >= 2^31 or a missing array, SPH_E_OOM when the
 * buffers cannot grow, SPH_E_CUDA for a launch or event failure. */
int sph_nsearch_run(sph_nsearch* ns, size_t n, const void* x, const void* y, const void* z,
                    double* stage_ms);

/* Copies the last run's sorted keys[n], permutation perm[n] (input index of each
 * sorted slot), cell_begin[ncell + 1] and sigma[n] (sorted order) to the host;
 * any pointer may be NULL.  Waits for the run. */
int sph_nsearch_results(sph_nsearch* ns, uint32_t* keys, uint32_t* perm, uint32_t* cell_begin,
                        double* sigma);

/* Cells of the grid (no synchronisation). */
size_t sph_nsearch_cell_count(const sph_nsearch* ns);

/* Frees everything (waits first). */
void sph_nsearch_destroy(sph_nsearch* ns);

/* ---- Decomposition of one tank into slabs: state by id range, schedule ----
 * A tank split into slabs along x (paper_2603_11868_gb300/slab.py) runs one
 * context per rank holding its own particles and ghost copies of its
 * neighbours' within a halo; after every acoustic step the ranks agree on the
 * velocity maximum and refresh the ghosts, and at every advection-step
 * boundary they hand over the particles that changed slab.  These calls move
 * that state; the paper has no counterpart (its runs are single-device).
 *
 * User ids are the indices of the last sph_set_particles(SPH_FLUID) call.
 * The state of user ids [id0, id0 + m) -- position and velocity (m x dim),
 * density, density rate (m), prior acceleration (m x dim), each a host array
 * in id order or NULL to skip it -- is copied out of the context / into it.
 * The density rate and the prior acceleration are held in the pair type
 * (float in mixed precision: values put are rounded to it).  Both calls
 * wait for the context's queued work.  SPH_E_INVALID when id0 + m > n,
 * SPH_E_STATE before fluid particles are set. */
int sph_get_state_range(sph_ctx* ctx, uint32_t id0, size_t m, double* pos, double* vel,
                        double* rho, double* drho, double* aprior);
int sph_put_state_range(sph_ctx* ctx, uint32_t id0, size_t m, const double* pos,
                        const double* vel, const double* rho, const double* drho,
                        const double* aprior);

/* Schedule scalars as eight doubles: t, tau (time since the advection step
 * began), dt_ad, dt_ac, acoustic steps, advection steps, started (0/1), and
 * the squared velocity maximum the next step's time steps come from.  get
 * reads them (waits); set writes them, and only where the next step begins
 * an advection step (tau >= dt_ad, or started = 0): SPH_E_INVALID otherwise
 * or for a negative or non-finite value.  set does not touch the particles. */
int sph_get_schedule(sph_ctx* ctx, double sched[8]);
int sph_set_schedule(sph_ctx* ctx, const double sched[8]);

/* max |v|^2 over the fluid particles whose user id is below n_own (a rank's
 * own particles, its ghosts excluded), into *vmax2.  Waits. */
int sph_owned_vmax2(sph_ctx* ctx, uint32_t n_own, double* vmax2);

/* Sets the squared velocity maximum the next step's time steps come from
 * (the ranks' common value, in place of the context's own).  Waits.
 * SPH_E_INVALID for a negative or non-finite value. */
int sph_set_vmax2(sph_ctx* ctx, double vmax2);

/* Device-memory forms of the per-step exchange, queued on the context's
 * stream in order with sph_step and returning without waiting (errors of the
 * queued work surface at the next waiting call), so that ghost refreshes and
 * the velocity maximum travel device to device (e.g. by NCCL on the same
 * stream):
 *   rows: m x (3 dim + 2) doubles per particle of user ids [id0, id0 + m):
 *         position, velocity, density, density rate, prior acceleration,
 *         caller-owned device memory (get writes them, put reads them);
 *   sph_owned_vmax2_device writes max |v|^2 of user ids below n_own as one
 *         double at device address vmax2 (non-negative doubles order like
 *         their 64-bit patterns, so an integer max-reduction of the bits
 *         combines ranks exactly);
 *   sph_set_vmax2_device reads the common value from device address vmax2.
 * SPH_E_INVALID for a bad range or NULL, SPH_E_STATE before fluid is set. */
int sph_get_state_rows_device(sph_ctx* ctx, uint32_t id0, size_t m, double* rows);
int sph_put_state_rows_device(sph_ctx* ctx, uint32_t id0, size_t m, const double* rows);
int sph_owned_vmax2_device(sph_ctx* ctx, uint32_t n_own, double* vmax2);
int sph_set_vmax2_device(sph_ctx* ctx, const double* vmax2);

/* Largest n accepted by sph_cell_sort_noalloc. */
#define SPH_NOALLOC_MAX_PARTICLES (1u << 20)

/* Cell sort that allocates no memory.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at the
 * moment they need a sort -- code that works inside a fixed memory budget
 * handed out in advance, code that must not stall the device (cudaMalloc and
 * cudaFree synchronise it), or code with no allocator at hand.
 *
 * It computes what sph_set_particles computes for the fluid: the cell key of
 * every particle on the grid of `domain` with cells of edge `cell_size` (pass
 * 2h to match a context), a stable sort of the particles by key (equal keys
 * keep the input order), and the CSR offsets of the cells.  All pointers are
 * device pointers:
 *   x, y, z         positions, n doubles each (z ignored, may be NULL, in 2D)
 *   keys_out[n]     sorted cell keys
 *   perm_out[n]     input index of each sorted slot
 *   cell_begin_out  ncell + 1 offsets, ncell = product of ceil((hi - lo) / cell_size)
 * Work is queued on `stream` (NULL = legacy default stream) and the call
 * returns without waiting.  Positions outside the domain are clamped into the
 * edge cell without an error report.
 *
 * Scratch memory: a file-scope device array sized for
 * SPH_NOALLOC_MAX_PARTICLES particles -- 2 * 2^20 + 256 * 256 + 256 words of
 * 4 bytes, 8 651 776 bytes (8.25 MiB) -- held on every GPU that loads the
 * library until the process exits.  n above that limit fails with
 * SPH_E_INVALID before any work is queued.  The first call on a device looks
 * up the array's device address and sets kernel attributes for that device
 * (the device must be current); make that first call before any stream
 * capture.  Those per-device settings are kept for the life of the process:
 * resetting the device (cudaDeviceReset) after the first call is not
 * supported.  No call allocates or frees memory.  All calls share the one
 * array, which keeps the previous call's contents (what must start at zero is
 * cleared by each call), so calls whose work overlaps on the GPU -- on
 * different streams, or from different threads -- race and corrupt each
 * other's results: order them on one stream or synchronise between them.
 * Returns SPH_OK, SPH_E_INVALID (bad arguments or n too large) or SPH_E_CUDA. */
int sph_cell_sort_noalloc(const sph_domain* domain, double cell_size, const double* x,
                          const double* y, const double* z, size_t n, uint32_t* keys_out,
                          uint32_t* perm_out, uint32_t* cell_begin_out, void* stream);

/* ---- Autotuner (the paper has no counterpart: it picks launch parameters
 * of this implementation).  A launch configuration: threads per block of the
 * neighbour loops (for a batch also the tile, the slots per work unit of its
 * persistent launches), the digit width of the radix sort, and whether the
 * loops walk neighbour lists.  None of them changes any result. */
typedef struct {
  int block;           /* SPH_OPT_BLOCK value */
  int radix_bits;      /* SPH_OPT_RADIX_BITS value */
  int neighbour_list;  /* SPH_OPT_NEIGHBOUR_LIST value */
  int trials;          /* configurations timed by the search */
  double ms_per_step;  /* measured device time per acoustic step */
} sph_tuning;

/* Picks the fastest configuration for this context as it stands: a
 * coordinate search (block size, then radix width, then lists on / off) in
 * which every candidate runs steps_per_trial acoustic steps (best of two
 * runs, CUDA-graph replay) from a device snapshot of the whole context; the
 * context is then restored to its state before the call and keeps the best
 * configuration, which is written to *best.  Needs device memory for the
 * snapshot (SPH_E_OOM otherwise); SPH_E_STATE before sph_set_particles. */
int sph_autotune(sph_ctx* ctx, int steps_per_trial, sph_tuning* best);

/* ---- Batches of independent tanks.  The paper runs one problem at a time;
 * a batch advances many small, independent problems together (each its own
 * domain, particles, material, gravity and its own dual-criteria schedule, so
 * its advection and acoustic steps have their own lengths).  Every stage of
 * an acoustic step is one persistent launch over the tiles of all tanks (the
 * rebuild stages over the tanks that begin an advection step in that step),
 * and the step is replayed as one CUDA graph.  A tank of a batch computes
 * exactly what an sph_ctx computes for it alone with the same options. */
typedef struct sph_batch sph_batch;

/* One tank: what sph_create takes for a single problem. */
typedef struct {
  sph_domain domain;
  double dp, h;
  sph_material material;
  double gravity[3];
} sph_tank;

/* Largest number of tanks in a batch. */
#define SPH_MAX_TANKS 1024

/* Creates a batch of n_tanks (1..SPH_MAX_TANKS) tanks, all of the same
 * dimension, computing in `precision`; allocator and stream as sph_create.
 * SPH_E_INVALID for a bad tank (same rules as sph_create) or a total cell
 * count of 2^31 or more. */
int sph_create_batch(int n_tanks, const sph_tank* tanks, int precision,
                     const sph_allocator* alloc, void* cuda_stream, sph_batch** out);

/* Sets the particles of one kind for every tank: counts[t] particles for
 * tank t (counts has n_tanks entries, a count may be 0), pos holds
 * sum(counts) * dim doubles, tank 0's particles first (vel, rho as
 * sph_set_particles: NULL = zero velocity / the tank's rho0; walls may take
 * prescribed sliding velocities, no density).  The total of each kind must
 * stay below 2^26. */
int sph_batch_set_particles(sph_batch* b, int kind, const size_t* counts, const double* pos,
                            const double* vel, const double* rho);

/* Queues n acoustic steps of every tank (each on its own schedule). */
int sph_batch_step(sph_batch* b, int n);

/* Fields as sph_get_fields, for all tanks: tank 0's particles first, each
 * tank in its user order. */
int sph_batch_get_fields(sph_batch* b, unsigned mask, double* out);

/* Schedule scalars of every tank (arrays of n_tanks; any may be NULL). */
int sph_batch_get_scalars(sph_batch* b, double* t, double* dt_ad, double* dt_ac, long* n_ac,
                          long* n_adv);

/* Neighbour structure of one tank after its last rebuild, in the tank's own
 * numbering (as sph_debug_neighbour_state for that tank alone): keys[n] the
 * binned cell of each storage slot, ids[n] the user index of each slot,
 * cell_begin[ncell + 1] (ncell of that tank's grid); any may be NULL. */
int sph_batch_debug_neighbour_state(sph_batch* b, int tank, uint32_t* keys, uint32_t* ids,
                                    uint32_t* cell_begin);

/* Totals over the tanks (kind = SPH_FLUID / SPH_WALL), the number of tanks,
 * and one tank's cell count (no synchronisation; 0 for a bad argument). */
size_t sph_batch_count(const sph_batch* b, int kind);
int sph_batch_tank_count(const sph_batch* b);
size_t sph_batch_cell_count(const sph_batch* b, int tank);

/* As sph_profile_stages / sph_kernels_per_step for a batch; rebuilds counts
 * the advection steps begun, summed over the tanks. */
int sph_batch_profile_stages(sph_batch* b, int n, double* ms, long* rebuilds);
long sph_batch_kernels_per_step(const sph_batch* b);

/* Options as sph_set_option (SPH_OPT_BLOCK also sets the tile: slots per
 * work unit of the persistent launches). */
int sph_batch_set_option(sph_batch* b, int option, long value);
int sph_batch_synchronize(sph_batch* b, double timeout_s);
const char* sph_batch_last_error(const sph_batch* b);
/* The autotuner of sph_autotune for a batch. */
int sph_batch_autotune(sph_batch* b, int steps_per_trial, sph_tuning* best);
void sph_batch_destroy(sph_batch* b);

/* Sets an sph_option; takes effect at the next sph_step. */
int sph_set_option(sph_ctx* ctx, int option, long value);

/* Waits for the context's queued work, giving up after timeout_s seconds
 * (<= 0: no limit) with SPH_E_TIMEOUT; the work is not cancelled.  Returns a
 * sticky device error if one was raised. */
int sph_synchronize(sph_ctx* ctx, double timeout_s);

/* Text of the last error on this context (never NULL; "" when none). */
const char* sph_last_error(const sph_ctx* ctx);

/* Frees the context and all its device memory (synchronises first). */
void sph_destroy(sph_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
