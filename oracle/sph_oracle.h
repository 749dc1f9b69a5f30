/*
 * Serial FP64 CPU oracle for the weakly-compressible SPH hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header or constant table with the CUDA library; the two are independent
 * restatements of the same method so that one can check the other.
 *
 * The method (the paper names the pieces; the equations are the published
 * SPHinXsys WCSPH forms, see the per-function comments in sph_oracle.c):
 *   - cell-linked list by cell key, stable sort, reorder and CSR cell offsets
 *     (paper, section "Cell linked-list, direct search and sorting");
 *   - direct search: kernel values recomputed from current positions for all
 *     particles of the 3^d neighbouring cells (same section);
 *   - Wendland C2 kernel, density summation with free-surface clamp,
 *     viscous force, Riemann-based pressure and density relaxation, static
 *     wall particles with a mirrored Riemann state, and the dual
 *     (advection / acoustic) time-step criteria.
 *
 * Layout conventions:
 *   positions / velocities passed in or out are n*dim doubles, particle-major
 *   (x0,y0[,z0],x1,...), in USER order (the order given to set_particles).
 */
#ifndef SPH_ORACLE_H
#define SPH_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct osim osim;

/* --- kernel function (Wendland C2) ------------------------------------- */
double osph_alpha(int dim, double h);
double osph_W(int dim, double h, double r);
double osph_dW(int dim, double h, double r);
/* reference number density: sum of W over an unperturbed lattice of spacing dp,
 * self included. */
double osph_sigma0(int dim, double dp, double h);

/* --- acoustic Riemann solver (fluid-fluid interface) ------------------- */
void osph_riemann(double pL, double pR, double rhoL, double rhoR, double UL,
                  double UR, double c0, double* Pstar, double* Ustar);

/* --- simulation ---------------------------------------------------------- */
osim* osph_create(int dim, const double lo[3], const double hi[3], double dp,
                  double h, double rho0, double c0, double mu, double U_ref,
                  const double g[3]);
void osph_destroy(osim* s);

/* kind 0 = fluid, 1 = wall.  vel / rho may be NULL (0 / rho0).  A wall's
 * vel is its prescribed velocity (NULL = at rest): the wall particles keep
 * their positions, so a nonzero velocity models a wall sliding along itself
 * (a lid, a belt, a Couette plate); it enters the mirrored Riemann state and
 * the viscous force.  Wall density is ignored.  Returns 0 on success. */
int osph_set_particles(osim* s, int kind, long n, const double* pos,
                       const double* vel, const double* rho);
/* translating walls (default none): moves[u] != 0 makes wall particle u
 * (user order of the last wall set) move with its velocity,
 * x_w(t) = x_w(0) + v_w t, t the simulation time; the other walls keep their
 * positions.  Translating walls are binned again at every rebuild and follow
 * the fluid's half-drifts: at t + dt/2 for the pressure relaxation, at
 * t + dt for the density relaxation.  NULL clears.  Returns 0. */
int osph_set_wall_translation(osim* s, const unsigned char* moves);
/* translating walls that also oscillate: wall u with moves[u] != 0 follows
 * x_w(t) = x_w(0) + v t + A sin(omega t) with A = amplitude[u * dim ..]
 * (NULL: none), so v_w = v + A omega cos(omega t), a_w = -A omega^2
 * sin(omega t); a_w enters the wall pressure p_w = p_i + rho_i
 * (x_w - x_i).(g - a_w).  osph_set_wall_translation is this call with no
 * amplitude.  Returns 0. */
int osph_set_wall_motion(osim* s, const unsigned char* moves, double omega,
                         const double* amplitude);
/* method variants: density_riemann = 1 (default) takes the Riemann U* in the
 * density relaxation, 0 the average of the two states; reinit_blended = 0
 * (default) reinitialises the density with the free-surface clamp
 * rho0 max(sigma / sigma0, 1), 1 with the blended form
 * rho_sum + max(0, rho_prev - rho_sum) rho0 / rho_prev. */
void osph_set_variant(osim* s, int density_riemann, int reinit_blended);

/* transport-velocity correction (default off): once per advection step,
 * after the density summation, fluid particles with sigma >= 0.95 sigma0 move
 * by -0.2 h^2 sum_j V_j grad_i W_ij (fluid V_j = m / rho_j, wall dp^dim) */
void osph_set_transport_correction(osim* s, int on);
void osph_transport_correction(osim* s);

/* set the carried density rate (user order, n values); default 0 */
int osph_set_drho(osim* s, const double* drho);
/* test infrastructure for slab-decomposed oracle runs: state of user ids
 * [id0, id0 + m) in / out (vectors m x 3), and the schedule scalars */
int osph_state_range(osim* s, long id0, long m, double* pos, double* vel, double* rho,
                     double* drho, double* aprior, int put);
void osph_set_schedule(osim* s, double t, double tau, double dt_ad, double dt_ac, long n_ac,
                       long n_adv, int started);

/* the full schedule: n acoustic steps */
int osph_step(osim* s, long n);

/* individual stages, for tests */
/* sets the simulation time (translating walls are placed and binned at it) */
void osph_set_time(osim* s, double t);
void osph_rebuild(osim* s);
void osph_density_summation(osim* s);
void osph_viscous(osim* s);
double osph_vmax2(const osim* s);
void osph_half1(osim* s, double dt);
void osph_pressure_relaxation(osim* s, double dt);
void osph_half2(osim* s, double dt);

/* field ids for osph_get_field */
enum {
  OSPH_POS = 0,    /* dim */
  OSPH_VEL = 1,    /* dim */
  OSPH_RHO = 2,    /* 1 */
  OSPH_P = 3,      /* 1 */
  OSPH_DRHO = 4,   /* 1 */
  OSPH_ACC = 5,    /* dim: pressure acceleration of the last pressure stage */
  OSPH_APRIOR = 6, /* dim: g + viscous acceleration */
  OSPH_SIGMA = 7   /* 1: kernel sum of the last density summation */
};
/* copy a field out in user order; returns the component count or -1 */
int osph_get_field(const osim* s, int field, double* out);

/* scalars: t, tau, dt_ad, dt_ac, then n_ac, n_adv, flags */
void osph_get_scalars(const osim* s, double* t, double* tau, double* dt_ad,
                      double* dt_ac, long* n_ac, long* n_adv, int* flags);
long osph_n(const osim* s);
long osph_nw(const osim* s);
long osph_ncell(const osim* s);
void osph_grid(const osim* s, double* cs, long nc[3]);

/* sorted state of the last rebuild (storage order): keys[n], perm[n]
 * (storage index k came from pre-sort index perm[k]), ids[n] (user id of
 * storage slot k), cell_begin[ncell+1].  Any pointer may be NULL. */
void osph_neighbour_state(const osim* s, uint32_t* keys, uint32_t* perm,
                          uint32_t* ids, uint32_t* cell_begin);
/* same for the wall set (sorted once, when set) */
void osph_wall_state(const osim* s, uint32_t* keys, uint32_t* ids,
                     uint32_t* cell_begin);

/* per fluid particle (user order): accepted fluid neighbours (self excluded),
 * accepted wall neighbours, and an order-free hash of the accepted ids.
 * brute = 1 scans all particles (O(N^2)) instead of the cell list. */
void osph_neighbour_stats(const osim* s, int brute, uint32_t* cnt_f,
                          uint32_t* cnt_w, uint64_t* hash);

/* diagnostics: surge front (max x over fluid) and kinetic energy */
void osph_front_ke(const osim* s, double* front, double* ke);

/* sampled evaluation at full size: for m fluid particles given by user id,
 * the kernel sum (density summation) with the current cell list. */
void osph_sample_sigma(const osim* s, long m, const uint32_t* user_ids,
                       double* sigma);
/* For a state as set (at rest, no carried density rate, binned): the pressure
 * acceleration the first acoustic step gives the m sampled fluid particles
 * (acc: m * dim). */
void osph_sample_first_step_acc(const osim* s, long m, const uint32_t* user_ids,
                                double* acc);

#ifdef __cplusplus
}
#endif
#endif
