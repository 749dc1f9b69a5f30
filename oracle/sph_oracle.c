/*
 * Serial FP64 CPU oracle for the weakly-compressible SPH hot path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, by the smoke check and by the
 * CPU-baseline leg of the benchmark, never by the product path.  Written to be
 * read against the method, not to be fast: one particle at a time, plain
 * loops, no blocking or fusion.  Build with -ffp-contract=off so that every
 * multiply and add is rounded on its own on every host.
 *
 * Sources.  The paper (Hu & Guarnieri, "Towards heterogeneous parallelism for
 * SPHinXsys") fixes the data-structure side: a cell-linked list built by
 * binning particles into cells of the cut-off size, particle sorting by cell
 * (radix sort on the device), and "direct search" in which every interaction
 * recomputes kernel values for all particles of the nearest cells (section
 * "Cell linked-list, direct search and sorting").  It gives no SPH equations;
 * the interactions follow the published SPHinXsys weakly-compressible method:
 *   [W95] Wendland C2 kernel,
 *   [Z17] Zhang, Hu & Adams, J. Comput. Phys. 335 (2017): Riemann-based
 *         pressure and density relaxation with a low-dissipation limiter,
 *   [Z20] Zhang, Hu & Adams, J. Comput. Phys. 404 (2020): dual-criteria
 *         (advection / acoustic) time stepping, density summation once per
 *         advection step, kick-drift-kick acoustic sub-steps.
 * Each reading the paper leaves open is stated where it is used.
 *
 * Pins (tests/test_oracle_*.py): kernel normalisation by quadrature, dW by
 * finite differences, lattice-sum convergence, brute-force neighbour sets,
 * sort invariants, Riemann special cases, momentum antisymmetry, reduction to
 * the textbook continuity / pressure-gradient / Laplacian forms, and the
 * hydrostatic column.
 */
#include "sph_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OSPH_PI 3.14159265358979323846

struct osim {
  int dim;
  double lo[3], hi[3], cs;
  long nc[3], ncell;
  double dp, h, rho0, c0, mu, U_ref, g[3];
  double V;      /* reference particle volume dp^dim (wall volume)        */
  double m;      /* fluid particle mass rho0 * V                           */
  double sigma0; /* lattice kernel sum: density summation normaliser        */

  /* fluid, storage order (sorted by cell at the last rebuild) */
  long n;
  double (*x)[3], (*v)[3], (*acc)[3], (*aprior)[3];
  double *rho, *drho, *p, *sigma;
  uint32_t *id, *key, *perm;
  long* cb; /* cell_begin, ncell + 1 entries */

  /* wall, sorted by cell: once, or at every rebuild when some walls
   * translate; vw, aw = wall velocity and acceleration at the current time
   * (zero at rest).  A wall slides along itself (fixed position, velocity
   * vwu) unless it translates: then it follows
   *   x_w(t) = x_w(0) + v t + A sin(omega t),
   *   v_w(t) = v + A omega cos(omega t),  a_w(t) = -A omega^2 sin(omega t),
   * v its given velocity, A its amplitude (zero: uniform motion).  xw0, vwu,
   * awu, wmoves keep the given positions, velocities, amplitudes and
   * translation flags in user order. */
  long nw;
  double (*xw)[3], (*vw)[3], (*aw)[3];
  uint32_t *idw, *keyw;
  long* cbw;
  double (*xw0)[3], (*vwu)[3], (*awu)[3];
  unsigned char* wmoves;
  int wtranslate; /* some wall translates */
  double womega;  /* angular frequency of the wall oscillation */

  double t, tau, dt_ad, dt_ac;
  long n_ac, n_adv;
  int started, flags;

  /* method variants (osph_set_variant) */
  int density_riemann; /* 1: Riemann U* in the density relaxation; 0: average */
  int reinit_blended;  /* 0: free-surface clamp; 1: blended reinitialisation */
  int transport;       /* 1: transport-velocity correction each advection step */
};

/* ------------------------------------------------------------------------ */
/* Wendland C2 kernel [W95]:  W(q) = alpha_d (1 - q/2)^4 (2q + 1),  q = r/h < 2,
 * alpha_2 = 7 / (4 pi h^2), alpha_3 = 21 / (16 pi h^3) (unit integral).     */
double osph_alpha(int dim, double h) {
  if (dim == 2) return 7.0 / (4.0 * OSPH_PI * h * h);
  return 21.0 / (16.0 * OSPH_PI * h * h * h);
}

double osph_W(int dim, double h, double r) {
  double q = r / h;
  if (q >= 2.0) return 0.0;
  double t = 1.0 - 0.5 * q;
  return osph_alpha(dim, h) * t * t * t * t * (2.0 * q + 1.0);
}

/* dW/dr = -5 alpha_d q (1 - q/2)^3 / h  (derivative of the form above) */
double osph_dW(int dim, double h, double r) {
  double q = r / h;
  if (q >= 2.0) return 0.0;
  double t = 1.0 - 0.5 * q;
  return -5.0 * osph_alpha(dim, h) * q * t * t * t / h;
}

/* Reference number density: kernel sum over the perfect lattice dp Z^d
 * centred on a particle, self included.  Density summation divides by it so
 * that an undisturbed interior lattice has rho = rho0 exactly (reading: the
 * paper is silent; SPHinXsys normalises by the lattice sum the same way). */
double osph_sigma0(int dim, double dp, double h) {
  int K = (int)ceil(2.0 * h / dp) + 1;
  int kz = dim == 3 ? K : 0;
  double s = 0.0;
  for (int c = -kz; c <= kz; ++c)
    for (int b = -K; b <= K; ++b)
      for (int a = -K; a <= K; ++a) {
        double r = dp * sqrt((double)(a * a + b * b + c * c));
        s += osph_W(dim, h, r);
      }
  return s;
}

/* Linearised acoustic Riemann problem between a left state (particle i) and
 * a right state (neighbour j) along the line from i to j [Z17]:
 *   rho_bar = (rhoL + rhoR) / 2, impedance rho_bar * c0 on both sides,
 *   beta    = min(3 max(UL - UR, 0) / c0, 1)    (low-dissipation limiter),
 *   P*      = (pL + pR)/2 + beta rho_bar c0 (UL - UR) / 2,
 *   U*      = (UL + UR)/2 + (pL - pR) / (2 rho_bar c0).                       */
void osph_riemann(double pL, double pR, double rhoL, double rhoR, double UL,
                  double UR, double c0, double* Pstar, double* Ustar) {
  double rho_bar = 0.5 * (rhoL + rhoR);
  double jump = UL - UR;
  double beta = 3.0 * (jump > 0.0 ? jump : 0.0) / c0;
  if (beta > 1.0) beta = 1.0;
  *Pstar = 0.5 * (pL + pR) + 0.5 * beta * rho_bar * c0 * jump;
  *Ustar = 0.5 * (UL + UR) + (pL - pR) / (2.0 * rho_bar * c0);
}

/* ------------------------------------------------------------------------ */
static void* xcalloc(size_t n, size_t sz) {
  void* p = calloc(n ? n : 1, sz);
  if (!p) abort();
  return p;
}

osim* osph_create(int dim, const double lo[3], const double hi[3], double dp,
                  double h, double rho0, double c0, double mu, double U_ref,
                  const double g[3]) {
  if (dim != 2 && dim != 3) return NULL;
  osim* s = (osim*)xcalloc(1, sizeof(osim));
  s->density_riemann = 1;
  s->dim = dim;
  s->dp = dp;
  s->h = h;
  s->rho0 = rho0;
  s->c0 = c0;
  s->mu = mu;
  s->U_ref = U_ref;
  /* cell size = cut-off radius 2h (paper: cells of the cut-off size) */
  s->cs = 2.0 * h;
  s->ncell = 1;
  for (int k = 0; k < 3; ++k) {
    s->g[k] = k < dim ? g[k] : 0.0;
    s->lo[k] = k < dim ? lo[k] : 0.0;
    s->hi[k] = k < dim ? hi[k] : 0.0;
    s->nc[k] = k < dim ? (long)ceil((hi[k] - lo[k]) / s->cs) : 1;
    if (s->nc[k] < 1) s->nc[k] = 1;
    s->ncell *= s->nc[k];
  }
  s->V = dim == 2 ? dp * dp : dp * dp * dp;
  s->m = rho0 * s->V;
  s->sigma0 = osph_sigma0(dim, dp, h);
  s->cb = (long*)xcalloc((size_t)s->ncell + 1, sizeof(long));
  s->cbw = (long*)xcalloc((size_t)s->ncell + 1, sizeof(long));
  return s;
}

static void free_fluid(osim* s) {
  free(s->x); free(s->v); free(s->acc); free(s->aprior);
  free(s->rho); free(s->drho); free(s->p); free(s->sigma);
  free(s->id); free(s->key); free(s->perm);
  s->x = s->v = s->acc = s->aprior = NULL;
  s->rho = s->drho = s->p = s->sigma = NULL;
  s->id = s->key = s->perm = NULL;
  s->n = 0;
}

void osph_destroy(osim* s) {
  if (!s) return;
  free_fluid(s);
  free(s->xw); free(s->vw); free(s->aw); free(s->idw); free(s->keyw);
  free(s->xw0); free(s->vwu); free(s->awu); free(s->wmoves);
  free(s->cb); free(s->cbw);
  free(s);
}

/* Cell key (paper: binning into cells of the cut-off size).
 *   c_k = floor((x_k - lo_k) / cs), clamped to [0, n_k - 1];
 *   key = (c_z n_y + c_y) n_x + c_x  (x fastest).
 * A coordinate outside the grid (or not finite) is clamped and flagged. */
static uint32_t cell_key(const osim* s, const double x[3], int* oob) {
  long c[3] = {0, 0, 0};
  for (int k = 0; k < s->dim; ++k) {
    double f = floor((x[k] - s->lo[k]) / s->cs);
    if (!(f >= 0.0)) {
      c[k] = 0;
      *oob = 1;
    } else if (f >= (double)s->nc[k]) {
      c[k] = s->nc[k] - 1;
      *oob = 1;
    } else {
      c[k] = (long)f;
    }
  }
  return (uint32_t)((c[2] * s->nc[1] + c[1]) * s->nc[0] + c[0]);
}

static void key_to_cell(const osim* s, uint32_t key, long c[3]) {
  long k = (long)key;
  c[0] = k % s->nc[0];
  k /= s->nc[0];
  c[1] = k % s->nc[1];
  c[2] = k / s->nc[1];
}

typedef struct {
  uint32_t key, idx;
} kv_t;

/* stable order: by key, ties by current storage position */
static int cmp_kv(const void* a, const void* b) {
  const kv_t* u = (const kv_t*)a;
  const kv_t* w = (const kv_t*)b;
  if (u->key != w->key) return u->key < w->key ? -1 : 1;
  if (u->idx != w->idx) return u->idx < w->idx ? -1 : 1;
  return 0;
}

/* cell_begin[c] = number of particles with key < c (CSR offsets) */
static void cell_offsets(const osim* s, const uint32_t* key, long n, long* cb) {
  for (long c = 0; c <= s->ncell; ++c) cb[c] = 0;
  for (long i = 0; i < n; ++i) cb[key[i] + 1] += 1;
  for (long c = 0; c < s->ncell; ++c) cb[c + 1] += cb[c];
}

static void permute3(double (*a)[3], const uint32_t* perm, long n) {
  double(*t)[3] = (double(*)[3])xcalloc((size_t)n, sizeof(double[3]));
  for (long k = 0; k < n; ++k)
    for (int d = 0; d < 3; ++d) t[k][d] = a[perm[k]][d];
  memcpy(a, t, (size_t)n * sizeof(double[3]));
  free(t);
}

static void permute1(double* a, const uint32_t* perm, long n) {
  double* t = (double*)xcalloc((size_t)n, sizeof(double));
  for (long k = 0; k < n; ++k) t[k] = a[perm[k]];
  memcpy(a, t, (size_t)n * sizeof(double));
  free(t);
}

static void permute_u(uint32_t* a, const uint32_t* perm, long n) {
  uint32_t* t = (uint32_t*)xcalloc((size_t)n, sizeof(uint32_t));
  for (long k = 0; k < n; ++k) t[k] = a[perm[k]];
  memcpy(a, t, (size_t)n * sizeof(uint32_t));
  free(t);
}

/* Position, velocity and acceleration of wall u (user order) at time t. */
static void wall_kinematics(const osim* s, uint32_t u, double t, double x[3], double v[3],
                            double a[3]) {
  const double sn = sin(s->womega * t), cs = cos(s->womega * t);
  for (int c = 0; c < 3; ++c) {
    if (s->wmoves[u]) {
      x[c] = s->xw0[u][c] + t * s->vwu[u][c] + s->awu[u][c] * sn;
      v[c] = s->vwu[u][c] + s->awu[u][c] * s->womega * cs;
      a[c] = -s->awu[u][c] * s->womega * s->womega * sn;
    } else {
      x[c] = s->xw0[u][c];
      v[c] = s->vwu[u][c];
      a[c] = 0.0;
    }
  }
}

/* Translating walls to time t (sorted slots, from the user-order copies). */
static void place_walls(osim* s, double t) {
  for (long k = 0; k < s->nw; ++k) {
    uint32_t u = s->idw[k];
    if (!s->wmoves[u]) continue;
    wall_kinematics(s, u, t, s->xw[k], s->vw[k], s->aw[k]);
  }
}

/* Bin the walls at time t: keys of their positions at t, a sort by key with
 * ties in user order, and the wall cell offsets. */
static void bin_walls(osim* s, double t) {
  long n = s->nw;
  kv_t* a = (kv_t*)xcalloc((size_t)(n > 0 ? n : 1), sizeof(kv_t));
  int oob = 0;
  for (long u = 0; u < n; ++u) {
    double xu[3], vu[3], au[3];
    wall_kinematics(s, (uint32_t)u, t, xu, vu, au);
    a[u].key = cell_key(s, xu, &oob);
    a[u].idx = (uint32_t)u;
  }
  if (oob) s->flags |= 1;
  qsort(a, (size_t)n, sizeof(kv_t), cmp_kv);
  for (long k = 0; k < n; ++k) {
    uint32_t u = a[k].idx;
    s->idw[k] = u;
    s->keyw[k] = a[k].key;
    wall_kinematics(s, u, t, s->xw[k], s->vw[k], s->aw[k]);
  }
  free(a);
  cell_offsets(s, s->keyw, n, s->cbw);
}

/* Rebuild of the cell-linked list: keys from the current FP64 positions, a
 * stable sort by key (ties keep the current storage order), reorder of every
 * per-particle field, and CSR cell offsets. */
void osph_rebuild(osim* s) {
  long n = s->n;
  kv_t* a = (kv_t*)xcalloc((size_t)n, sizeof(kv_t));
  int oob = 0;
  for (long i = 0; i < n; ++i) {
    a[i].key = cell_key(s, s->x[i], &oob);
    a[i].idx = (uint32_t)i;
  }
  if (oob) s->flags |= 1;
  qsort(a, (size_t)n, sizeof(kv_t), cmp_kv);
  for (long k = 0; k < n; ++k) {
    s->perm[k] = a[k].idx;
    s->key[k] = a[k].key;
  }
  free(a);
  permute3(s->x, s->perm, n);
  permute3(s->v, s->perm, n);
  permute3(s->acc, s->perm, n);
  permute3(s->aprior, s->perm, n);
  permute1(s->rho, s->perm, n);
  permute1(s->drho, s->perm, n);
  permute1(s->p, s->perm, n);
  permute1(s->sigma, s->perm, n);
  permute_u(s->id, s->perm, n);
  cell_offsets(s, s->key, n, s->cb);
  /* translating walls are binned again at the rebuild time */
  if (s->wtranslate) bin_walls(s, s->t);
}

int osph_set_wall_motion(osim* s, const unsigned char* moves, double omega,
                         const double* amplitude) {
  const int d = s->dim;
  s->wtranslate = 0;
  s->womega = omega;
  for (long u = 0; u < s->nw; ++u) {
    s->wmoves[u] = moves ? (moves[u] ? 1 : 0) : 0;
    if (s->wmoves[u]) s->wtranslate = 1;
    for (int c = 0; c < 3; ++c) s->awu[u][c] = (amplitude && c < d) ? amplitude[u * d + c] : 0.0;
  }
  bin_walls(s, s->t);
  return 0;
}

void osph_set_time(osim* s, double t) {
  s->t = t;
  if (s->wtranslate) bin_walls(s, t);
}

int osph_set_wall_translation(osim* s, const unsigned char* moves) {
  return osph_set_wall_motion(s, moves, 0.0, NULL);
}

int osph_set_particles(osim* s, int kind, long n, const double* pos,
                       const double* vel, const double* rho) {
  int d = s->dim;
  if (n < 0) return 1;
  if (kind == 0) {
    free_fluid(s);
    s->n = n;
    s->x = (double(*)[3])xcalloc((size_t)n, sizeof(double[3]));
    s->v = (double(*)[3])xcalloc((size_t)n, sizeof(double[3]));
    s->acc = (double(*)[3])xcalloc((size_t)n, sizeof(double[3]));
    s->aprior = (double(*)[3])xcalloc((size_t)n, sizeof(double[3]));
    s->rho = (double*)xcalloc((size_t)n, sizeof(double));
    s->drho = (double*)xcalloc((size_t)n, sizeof(double));
    s->p = (double*)xcalloc((size_t)n, sizeof(double));
    s->sigma = (double*)xcalloc((size_t)n, sizeof(double));
    s->id = (uint32_t*)xcalloc((size_t)n, sizeof(uint32_t));
    s->key = (uint32_t*)xcalloc((size_t)n, sizeof(uint32_t));
    s->perm = (uint32_t*)xcalloc((size_t)n, sizeof(uint32_t));
    for (long i = 0; i < n; ++i) {
      for (int k = 0; k < d; ++k) {
        s->x[i][k] = pos[i * d + k];
        s->v[i][k] = vel ? vel[i * d + k] : 0.0;
      }
      s->rho[i] = rho ? rho[i] : s->rho0;
      s->p[i] = s->c0 * s->c0 * (s->rho[i] - s->rho0);
      s->id[i] = (uint32_t)i;
      s->perm[i] = (uint32_t)i;
    }
    s->started = 0;
    s->t = s->tau = s->dt_ad = s->dt_ac = 0.0;
    s->n_ac = s->n_adv = 0;
    s->flags = 0;
    /* bin once so that stages can be called before the first step */
    osph_rebuild(s);
    return 0;
  }
  if (kind == 1) {
    free(s->xw); free(s->vw); free(s->aw); free(s->idw); free(s->keyw);
    free(s->xw0); free(s->vwu); free(s->awu); free(s->wmoves);
    s->nw = n;
    s->xw = (double(*)[3])xcalloc((size_t)n, sizeof(double[3]));
    s->vw = (double(*)[3])xcalloc((size_t)n, sizeof(double[3]));
    s->aw = (double(*)[3])xcalloc((size_t)n, sizeof(double[3]));
    s->idw = (uint32_t*)xcalloc((size_t)n, sizeof(uint32_t));
    s->keyw = (uint32_t*)xcalloc((size_t)n, sizeof(uint32_t));
    s->xw0 = (double(*)[3])xcalloc((size_t)n, sizeof(double[3]));
    s->vwu = (double(*)[3])xcalloc((size_t)n, sizeof(double[3]));
    s->awu = (double(*)[3])xcalloc((size_t)n, sizeof(double[3]));
    s->wmoves = (unsigned char*)xcalloc((size_t)n, 1);
    s->wtranslate = 0;
    s->womega = 0.0;
    for (long i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) {
        s->xw0[i][c] = c < d ? pos[i * d + c] : 0.0;
        s->vwu[i][c] = (c < d && vel) ? vel[i * d + c] : 0.0;
      }
    bin_walls(s, 0.0);
    return 0;
  }
  return 1;
}

int osph_set_drho(osim* s, const double* drho) {
  for (long k = 0; k < s->n; ++k) s->drho[k] = drho[s->id[k]];
  return 0;
}

/* State of the fluid particles with user ids [id0, id0 + m), arrays in id
 * order (position, velocity and prior acceleration m x 3 with the unused
 * components 0; NULL skips a field): copied in (put) or out.  Test
 * infrastructure for running the oracle as the ranks of a slab
 * decomposition; no arithmetic of the method. */
int osph_state_range(osim* s, long id0, long m, double* pos, double* vel, double* rho,
                     double* drho, double* aprior, int put) {
  if (id0 < 0 || m < 0 || id0 + m > s->n) return 1;
  for (long k = 0; k < s->n; ++k) {
    long u = (long)s->id[k] - id0;
    if (u < 0 || u >= m) continue;
    for (int c = 0; c < 3; ++c) {
      if (pos) { if (put) s->x[k][c] = pos[u * 3 + c]; else pos[u * 3 + c] = s->x[k][c]; }
      if (vel) { if (put) s->v[k][c] = vel[u * 3 + c]; else vel[u * 3 + c] = s->v[k][c]; }
      if (aprior) {
        if (put) s->aprior[k][c] = aprior[u * 3 + c];
        else aprior[u * 3 + c] = s->aprior[k][c];
      }
    }
    if (rho) { if (put) s->rho[k] = rho[u]; else rho[u] = s->rho[k]; }
    if (drho) { if (put) s->drho[k] = drho[u]; else drho[u] = s->drho[k]; }
  }
  return 0;
}

/* The schedule scalars t, tau, dt_ad, dt_ac, acoustic and advection step
 * counts and the started flag (test infrastructure, as above). */
void osph_set_schedule(osim* s, double t, double tau, double dt_ad, double dt_ac, long n_ac,
                       long n_adv, int started) {
  s->t = t;
  s->tau = tau;
  s->dt_ad = dt_ad;
  s->dt_ac = dt_ac;
  s->n_ac = n_ac;
  s->n_adv = n_adv;
  s->started = started;
}

/* The 3^d cells around a binned cell, in the order dz, dy, dx = -1..1,
 * skipping cells outside the grid. */
static int neighbour_cells(const osim* s, uint32_t key, long* out) {
  long c[3];
  key_to_cell(s, key, c);
  int kz = s->dim == 3 ? 1 : 0;
  int m = 0;
  for (int dz = -kz; dz <= kz; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        long a = c[0] + dx, b = c[1] + dy, z = c[2] + dz;
        if (a < 0 || a >= s->nc[0] || b < 0 || b >= s->nc[1] || z < 0 ||
            z >= s->nc[2])
          continue;
        out[m++] = (z * s->nc[1] + b) * s->nc[0] + a;
      }
  return m;
}

static double dist2(const double a[3], const double b[3]) {
  double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
  return d0 * d0 + d1 * d1 + d2 * d2;
}

/* Density summation (once per advection step) [Z20]:
 *   sigma_i = sum_{j in fluid and wall, r_ij < 2h} W(r_ij)   (self included),
 *   rho_i   = rho0 * max(sigma_i / sigma0, 1)    (reading: free-surface clamp),
 *   p_i     = c0^2 (rho_i - rho0).                                         */
static double sigma_of(const osim* s, long i) {
  const double r2max = 4.0 * s->h * s->h;
  long cells[27];
  int nc = neighbour_cells(s, s->key[i], cells);
  double sig = 0.0;
  for (int q = 0; q < nc; ++q) {
    for (long j = s->cb[cells[q]]; j < s->cb[cells[q] + 1]; ++j) {
      double r2 = dist2(s->x[i], s->x[j]);
      if (r2 >= r2max) continue;
      sig += osph_W(s->dim, s->h, sqrt(r2));
    }
    for (long w = s->cbw[cells[q]]; w < s->cbw[cells[q] + 1]; ++w) {
      double r2 = dist2(s->x[i], s->xw[w]);
      if (r2 >= r2max) continue;
      sig += osph_W(s->dim, s->h, sqrt(r2));
    }
  }
  return sig;
}

static double density_of_sigma(const osim* s, double sig) {
  double ratio = sig / s->sigma0;
  return s->rho0 * (ratio > 1.0 ? ratio : 1.0);
}

/* Blended free-surface reinitialisation (variant; SPHinXsys free-surface
 * density summation): with rho_sum = rho0 sigma / sigma0 and the density
 * carried into the summation rho_prev,
 *   rho = rho_sum + max(0, rho_prev - rho_sum) rho0 / rho_prev,
 * so a particle with full kernel support (rho_sum >= rho_prev) takes the
 * summed density and a particle near the surface keeps part of its own. */
static double density_blended(const osim* s, double sig, double rho_prev) {
  double rho_sum = s->rho0 * (sig / s->sigma0);
  double excess = rho_prev - rho_sum;
  return rho_sum + (excess > 0.0 ? excess : 0.0) * s->rho0 / rho_prev;
}

void osph_density_summation(osim* s) {
  for (long i = 0; i < s->n; ++i) s->sigma[i] = sigma_of(s, i);
  for (long i = 0; i < s->n; ++i) {
    s->rho[i] = s->reinit_blended ? density_blended(s, s->sigma[i], s->rho[i])
                                  : density_of_sigma(s, s->sigma[i]);
    s->p[i] = s->c0 * s->c0 * (s->rho[i] - s->rho0);
  }
}

void osph_set_variant(osim* s, int density_riemann, int reinit_blended) {
  s->density_riemann = density_riemann ? 1 : 0;
  s->reinit_blended = reinit_blended ? 1 : 0;
}

/* Viscous force (once per advection step), SPHinXsys form:
 *   a_prior_i = g + (2 mu / rho_i) sum_j V_j (v_i - v_j) W'(r_ij) / (r_ij + 0.01 h)
 * with V_j = m / rho_j for fluid.  A wall particle (V_w = dp^d) enters with
 * the mirrored velocity v_R = 2 v_w - v_i of the Riemann wall state in place
 * of v_j (v_w its prescribed velocity, 0 at rest), so its pair term carries
 * v_i - v_R = 2 (v_i - v_w): the velocity interpolated half-way between the
 * fluid particle and its image is v_w, the no-slip condition at the wall
 * surface (reading; the simpler v_j = v_w gives the wall half that weight and
 * lets the fluid slip).  Self is excluded (r = 0 contributes nothing). */
void osph_viscous(osim* s) {
  const double r2max = 4.0 * s->h * s->h;
  const double eps = 0.01 * s->h;
  long cells[27];
  for (long i = 0; i < s->n; ++i) {
    int nc = neighbour_cells(s, s->key[i], cells);
    double a[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < nc; ++q) {
      for (long j = s->cb[cells[q]]; j < s->cb[cells[q] + 1]; ++j) {
        if (j == i) continue;
        double r2 = dist2(s->x[i], s->x[j]);
        if (r2 >= r2max) continue;
        double r = sqrt(r2);
        double coef = (s->m / s->rho[j]) * osph_dW(s->dim, s->h, r) / (r + eps);
        for (int k = 0; k < 3; ++k) a[k] += coef * (s->v[i][k] - s->v[j][k]);
      }
      for (long w = s->cbw[cells[q]]; w < s->cbw[cells[q] + 1]; ++w) {
        double r2 = dist2(s->x[i], s->xw[w]);
        if (r2 >= r2max) continue;
        double r = sqrt(r2);
        double coef = s->V * osph_dW(s->dim, s->h, r) / (r + eps);
        for (int k = 0; k < 3; ++k) a[k] += coef * (2.0 * (s->v[i][k] - s->vw[w][k]));
      }
    }
    for (int k = 0; k < 3; ++k)
      s->aprior[i][k] = s->g[k] + 2.0 * s->mu / s->rho[i] * a[k];
  }
}

/* Transport-velocity (particle-shifting) correction (variant, a reading of
 * SPHinXsys's transport velocity correction): once per advection step,
 * right after the density summation, every fluid particle whose kernel sum
 * shows full support (sigma_i >= 0.95 sigma0) moves by
 *   dr_i = -C h^2 sum_j V_j W'(r_ij) e_ij,   C = 0.2,
 * over its fluid (V_j = m / rho_j) and wall (V_w = dp^d) neighbours, self
 * excluded.  All shifts come from the positions before any is applied.  The
 * sum is the SPH gradient of the particle concentration, so the shift moves a
 * particle from crowded towards sparse neighbourhoods. */
void osph_transport_correction(osim* s) {
  const double r2max = 4.0 * s->h * s->h;
  const double coef = -0.2 * s->h * s->h;
  double (*d)[3] = (double (*)[3])xcalloc((size_t)(s->n > 0 ? s->n : 1), sizeof *d);
  long cells[27];
  for (long i = 0; i < s->n; ++i) {
    if (s->sigma[i] < 0.95 * s->sigma0) continue;
    int nc = neighbour_cells(s, s->key[i], cells);
    double g[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < nc; ++q) {
      for (long j = s->cb[cells[q]]; j < s->cb[cells[q] + 1]; ++j) {
        if (j == i) continue;
        double r2 = dist2(s->x[i], s->x[j]);
        if (r2 >= r2max) continue;
        double r = sqrt(r2);
        double f = (s->m / s->rho[j]) * osph_dW(s->dim, s->h, r) / r;
        for (int k = 0; k < 3; ++k) g[k] += f * (s->x[i][k] - s->x[j][k]);
      }
      for (long w = s->cbw[cells[q]]; w < s->cbw[cells[q] + 1]; ++w) {
        double r2 = dist2(s->x[i], s->xw[w]);
        if (r2 >= r2max) continue;
        double r = sqrt(r2);
        double f = s->V * osph_dW(s->dim, s->h, r) / r;
        for (int k = 0; k < 3; ++k) g[k] += f * (s->x[i][k] - s->xw[w][k]);
      }
    }
    for (int k = 0; k < 3; ++k) d[i][k] = coef * g[k];
  }
  for (long i = 0; i < s->n; ++i)
    for (int k = 0; k < s->dim; ++k) s->x[i][k] += d[i][k];
  free(d);
}

void osph_set_transport_correction(osim* s, int on) { s->transport = on ? 1 : 0; }

double osph_vmax2(const osim* s) {
  double m = 0.0;
  for (long i = 0; i < s->n; ++i) {
    double u = s->v[i][0] * s->v[i][0] + s->v[i][1] * s->v[i][1] +
               s->v[i][2] * s->v[i][2];
    if (u > m) m = u;
  }
  return m;
}

/* First half of the acoustic step [Z17]: density by the carried rate, pressure
 * by the linear equation of state, positions by half a step (translating
 * walls to t + dt/2). */
void osph_half1(osim* s, double dt) {
  for (long i = 0; i < s->n; ++i) {
    s->rho[i] += 0.5 * dt * s->drho[i];
    s->p[i] = s->c0 * s->c0 * (s->rho[i] - s->rho0);
    for (int k = 0; k < s->dim; ++k) s->x[i][k] += 0.5 * dt * s->v[i][k];
  }
  /* translating walls follow to the same time (reading) */
  if (s->wtranslate) place_walls(s, s->t + 0.5 * dt);
}

/* Riemann-based pressure relaxation [Z17], then the velocity kick.
 * For the pair (i, j): e_ij = (x_i - x_j) / r_ij, U_L = -v_i.e_ij,
 * U_R = -v_j.e_ij, and
 *   a_i = -(2 / rho_i) sum_j P*_ij V_j W'(r_ij) e_ij,   V_j = m / rho_j.
 * Wall particle w (velocity v_w and acceleration a_w at the current time:
 * zero at rest, v_w for a sliding wall, both for a translating one) supplies
 * a mirrored right state (reading: pressure extrapolated along the effective
 * gravity of the wall's frame, density from the inverse equation of state
 * and volume from that density, as in Adami, Hu & Adams, J. Comput. Phys.
 * 231 (2012)):
 *   p_w = p_i + rho_i (x_w - x_i).(g - a_w),  rho_w = rho0 + p_w / c0^2,
 *   v_R = 2 v_w - v_i,  V_w = m / rho_w.
 * Then v_i += dt (a_i + a_prior_i). */
/* Pressure acceleration of storage slot i with the given density and
 * pressure arrays (indexed by storage slot). */
/* v_R . e for the mirrored wall state v_R = 2 v_w - v_i */
static double mirror_dot(const double vi[3], const double vw[3], const double e[3]) {
  double d = 0.0;
  for (int k = 0; k < 3; ++k) d += (2.0 * vw[k] - vi[k]) * e[k];
  return d;
}

static void pressure_acc_of(const osim* s, long i, const double* rho, const double* p,
                            double out[3]) {
  const double r2max = 4.0 * s->h * s->h;
  const double c0 = s->c0;
  long cells[27];
  int nc = neighbour_cells(s, s->key[i], cells);
  double a[3] = {0.0, 0.0, 0.0};
  for (int q = 0; q < nc; ++q) {
    for (long j = s->cb[cells[q]]; j < s->cb[cells[q] + 1]; ++j) {
      if (j == i) continue;
      double r2 = dist2(s->x[i], s->x[j]);
      if (r2 >= r2max) continue;
      double r = sqrt(r2);
      double e[3];
      for (int k = 0; k < 3; ++k) e[k] = (s->x[i][k] - s->x[j][k]) / r;
      double UL = -(s->v[i][0] * e[0] + s->v[i][1] * e[1] + s->v[i][2] * e[2]);
      double UR = -(s->v[j][0] * e[0] + s->v[j][1] * e[1] + s->v[j][2] * e[2]);
      double Ps, Us;
      osph_riemann(p[i], p[j], rho[i], rho[j], UL, UR, c0, &Ps, &Us);
      double f = Ps * (s->m / rho[j]) * osph_dW(s->dim, s->h, r);
      for (int k = 0; k < 3; ++k) a[k] += f * e[k];
    }
    for (long w = s->cbw[cells[q]]; w < s->cbw[cells[q] + 1]; ++w) {
      double r2 = dist2(s->x[i], s->xw[w]);
      if (r2 >= r2max) continue;
      double r = sqrt(r2);
      double e[3];
      for (int k = 0; k < 3; ++k) e[k] = (s->x[i][k] - s->xw[w][k]) / r;
      double gdot = 0.0;
      for (int k = 0; k < 3; ++k) gdot += (s->xw[w][k] - s->x[i][k]) * (s->g[k] - s->aw[w][k]);
      double pw = p[i] + rho[i] * gdot;
      double rhow = s->rho0 + pw / (c0 * c0);
      double UL = -(s->v[i][0] * e[0] + s->v[i][1] * e[1] + s->v[i][2] * e[2]);
      double UR = -mirror_dot(s->v[i], s->vw[w], e);
      double Ps, Us;
      osph_riemann(p[i], pw, rho[i], rhow, UL, UR, c0, &Ps, &Us);
      double f = Ps * (s->m / rhow) * osph_dW(s->dim, s->h, r);
      for (int k = 0; k < 3; ++k) a[k] += f * e[k];
    }
  }
  for (int k = 0; k < 3; ++k) out[k] = -2.0 / rho[i] * a[k];
}

/* Riemann-based pressure relaxation [Z17], then the velocity kick.
 * For the pair (i, j): e_ij = (x_i - x_j) / r_ij, U_L = -v_i.e_ij,
 * U_R = -v_j.e_ij, and
 *   a_i = -(2 / rho_i) sum_j P*_ij V_j W'(r_ij) e_ij,   V_j = m / rho_j.
 * Wall particle w (static, v_w = 0) supplies a mirrored right state
 * (reading: pressure extrapolated along gravity, density from the inverse
 * equation of state and volume from that density, as in Adami, Hu & Adams,
 * J. Comput. Phys. 231 (2012)):
 *   p_w = p_i + rho_i (x_w - x_i).g,  rho_w = rho0 + p_w / c0^2,
 *   v_R = 2 v_w - v_i = -v_i,  V_w = m / rho_w.
 * Then v_i += dt (a_i + a_prior_i). */
void osph_pressure_relaxation(osim* s, double dt) {
  for (long i = 0; i < s->n; ++i) pressure_acc_of(s, i, s->rho, s->p, s->acc[i]);
  for (long i = 0; i < s->n; ++i)
    for (int k = 0; k < s->dim; ++k)
      s->v[i][k] += dt * (s->acc[i][k] + s->aprior[i][k]);
}

/* Second half of the acoustic step [Z17]: positions by half a step
 * (translating walls to t + dt), then the
 * Riemann-based density relaxation
 *   drho_i = -2 rho_i sum_j V_j W'(r_ij) (U_L - U*_ij)
 * (fluid V_j = m / rho_j; wall: mirrored state and V_w = m / rho_w as in
 * the pressure stage), then rho_i += dt/2 drho_i.
 * Variant without the Riemann solver (density_riemann = 0): U* is the plain
 * average (U_L + U_R) / 2, which makes this the textbook SPH continuity
 * equation drho_i = rho_i sum_j V_j W'(r_ij) (v_i - v_j).e_ij. */
void osph_half2(osim* s, double dt) {
  const double r2max = 4.0 * s->h * s->h;
  const double c0 = s->c0;
  long cells[27];
  for (long i = 0; i < s->n; ++i)
    for (int k = 0; k < s->dim; ++k) s->x[i][k] += 0.5 * dt * s->v[i][k];
  if (s->wtranslate) place_walls(s, s->t + dt);
  for (long i = 0; i < s->n; ++i) {
    int nc = neighbour_cells(s, s->key[i], cells);
    double sum = 0.0;
    for (int q = 0; q < nc; ++q) {
      for (long j = s->cb[cells[q]]; j < s->cb[cells[q] + 1]; ++j) {
        if (j == i) continue;
        double r2 = dist2(s->x[i], s->x[j]);
        if (r2 >= r2max) continue;
        double r = sqrt(r2);
        double e[3];
        for (int k = 0; k < 3; ++k) e[k] = (s->x[i][k] - s->x[j][k]) / r;
        double UL = -(s->v[i][0] * e[0] + s->v[i][1] * e[1] + s->v[i][2] * e[2]);
        double UR = -(s->v[j][0] * e[0] + s->v[j][1] * e[1] + s->v[j][2] * e[2]);
        double Ps, Us;
        osph_riemann(s->p[i], s->p[j], s->rho[i], s->rho[j], UL, UR, c0, &Ps, &Us);
        if (!s->density_riemann) Us = 0.5 * (UL + UR);
        sum += (s->m / s->rho[j]) * osph_dW(s->dim, s->h, r) * (UL - Us);
      }
      for (long w = s->cbw[cells[q]]; w < s->cbw[cells[q] + 1]; ++w) {
        double r2 = dist2(s->x[i], s->xw[w]);
        if (r2 >= r2max) continue;
        double r = sqrt(r2);
        double e[3];
        for (int k = 0; k < 3; ++k) e[k] = (s->x[i][k] - s->xw[w][k]) / r;
        double gdot = 0.0;
        for (int k = 0; k < 3; ++k)
          gdot += (s->xw[w][k] - s->x[i][k]) * (s->g[k] - s->aw[w][k]);
        double pw = s->p[i] + s->rho[i] * gdot;
        double rhow = s->rho0 + pw / (c0 * c0);
        double UL = -(s->v[i][0] * e[0] + s->v[i][1] * e[1] + s->v[i][2] * e[2]);
        double UR = -mirror_dot(s->v[i], s->vw[w], e);
        double Ps, Us;
        osph_riemann(s->p[i], pw, s->rho[i], rhow, UL, UR, c0, &Ps, &Us);
        if (!s->density_riemann) Us = 0.5 * (UL + UR);
        sum += (s->m / rhow) * osph_dW(s->dim, s->h, r) * (UL - Us);
      }
    }
    s->drho[i] = -2.0 * s->rho[i] * sum;
  }
  for (long i = 0; i < s->n; ++i) s->rho[i] += 0.5 * dt * s->drho[i];
}

/* Dual-criteria schedule [Z20].  Per acoustic step:
 *   Vmax^2 = max_i |v_i|^2;
 *   if this is the first step or tau >= dt_ad, an advection step begins:
 *       dt_ad = 0.25 h / max(U_ref, Vmax); rebuild; density summation;
 *       viscous force; tau = 0;
 *   dt_ac = 0.6 h / (c0 + Vmax);
 *   half1, pressure relaxation, half2;  t += dt_ac, tau += dt_ac.
 * (Reading: no clipping of the last acoustic step to the advection step.) */
int osph_step(osim* s, long nsteps) {
  for (long k = 0; k < nsteps; ++k) {
    double vmax = sqrt(osph_vmax2(s));
    if (!s->started || s->tau >= s->dt_ad) {
      s->dt_ad = 0.25 * s->h / (s->U_ref > vmax ? s->U_ref : vmax);
      osph_rebuild(s);
      osph_density_summation(s);
      if (s->transport) osph_transport_correction(s);
      osph_viscous(s);
      s->tau = 0.0;
      s->n_adv += 1;
      s->started = 1;
    }
    s->dt_ac = 0.6 * s->h / (s->c0 + vmax);
    osph_half1(s, s->dt_ac);
    osph_pressure_relaxation(s, s->dt_ac);
    osph_half2(s, s->dt_ac);
    s->t += s->dt_ac;
    s->tau += s->dt_ac;
    s->n_ac += 1;
  }
  return s->flags;
}

/* ------------------------------------------------------------------------ */
int osph_get_field(const osim* s, int field, double* out) {
  int d = s->dim;
  for (long k = 0; k < s->n; ++k) {
    long u = s->id[k];
    switch (field) {
      case OSPH_POS: for (int c = 0; c < d; ++c) out[u * d + c] = s->x[k][c]; break;
      case OSPH_VEL: for (int c = 0; c < d; ++c) out[u * d + c] = s->v[k][c]; break;
      case OSPH_ACC: for (int c = 0; c < d; ++c) out[u * d + c] = s->acc[k][c]; break;
      case OSPH_APRIOR: for (int c = 0; c < d; ++c) out[u * d + c] = s->aprior[k][c]; break;
      case OSPH_RHO: out[u] = s->rho[k]; break;
      case OSPH_P: out[u] = s->p[k]; break;
      case OSPH_DRHO: out[u] = s->drho[k]; break;
      case OSPH_SIGMA: out[u] = s->sigma[k]; break;
      default: return -1;
    }
  }
  if (field == OSPH_POS || field == OSPH_VEL || field == OSPH_ACC || field == OSPH_APRIOR)
    return d;
  return 1;
}

void osph_get_scalars(const osim* s, double* t, double* tau, double* dt_ad,
                      double* dt_ac, long* n_ac, long* n_adv, int* flags) {
  if (t) *t = s->t;
  if (tau) *tau = s->tau;
  if (dt_ad) *dt_ad = s->dt_ad;
  if (dt_ac) *dt_ac = s->dt_ac;
  if (n_ac) *n_ac = s->n_ac;
  if (n_adv) *n_adv = s->n_adv;
  if (flags) *flags = s->flags;
}

long osph_n(const osim* s) { return s->n; }
long osph_nw(const osim* s) { return s->nw; }
long osph_ncell(const osim* s) { return s->ncell; }
void osph_grid(const osim* s, double* cs, long nc[3]) {
  *cs = s->cs;
  for (int k = 0; k < 3; ++k) nc[k] = s->nc[k];
}

void osph_neighbour_state(const osim* s, uint32_t* keys, uint32_t* perm,
                          uint32_t* ids, uint32_t* cell_begin) {
  for (long k = 0; k < s->n; ++k) {
    if (keys) keys[k] = s->key[k];
    if (perm) perm[k] = s->perm[k];
    if (ids) ids[k] = s->id[k];
  }
  if (cell_begin)
    for (long c = 0; c <= s->ncell; ++c) cell_begin[c] = (uint32_t)s->cb[c];
}

void osph_wall_state(const osim* s, uint32_t* keys, uint32_t* ids,
                     uint32_t* cell_begin) {
  for (long k = 0; k < s->nw; ++k) {
    if (keys) keys[k] = s->keyw[k];
    if (ids) ids[k] = s->idw[k];
  }
  if (cell_begin)
    for (long c = 0; c <= s->ncell; ++c) cell_begin[c] = (uint32_t)s->cbw[c];
}

/* SplitMix64 output function (Steele, Lea & Flood 2014), used as an
 * order-free fingerprint of a neighbour set. */
static uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

void osph_neighbour_stats(const osim* s, int brute, uint32_t* cnt_f,
                          uint32_t* cnt_w, uint64_t* hash) {
  const double r2max = 4.0 * s->h * s->h;
  long cells[27];
  for (long i = 0; i < s->n; ++i) {
    uint32_t nf = 0, nw = 0;
    uint64_t hs = 0;
    if (brute) {
      for (long j = 0; j < s->n; ++j) {
        if (j == i || dist2(s->x[i], s->x[j]) >= r2max) continue;
        nf++;
        hs += mix64(s->id[j]);
      }
      for (long w = 0; w < s->nw; ++w) {
        if (dist2(s->x[i], s->xw[w]) >= r2max) continue;
        nw++;
        hs += mix64((1ULL << 40) + s->idw[w]);
      }
    } else {
      int nc = neighbour_cells(s, s->key[i], cells);
      for (int q = 0; q < nc; ++q) {
        for (long j = s->cb[cells[q]]; j < s->cb[cells[q] + 1]; ++j) {
          if (j == i || dist2(s->x[i], s->x[j]) >= r2max) continue;
          nf++;
          hs += mix64(s->id[j]);
        }
        for (long w = s->cbw[cells[q]]; w < s->cbw[cells[q] + 1]; ++w) {
          if (dist2(s->x[i], s->xw[w]) >= r2max) continue;
          nw++;
          hs += mix64((1ULL << 40) + s->idw[w]);
        }
      }
    }
    long u = s->id[i];
    if (cnt_f) cnt_f[u] = nf;
    if (cnt_w) cnt_w[u] = nw;
    if (hash) hash[u] = hs;
  }
}

void osph_front_ke(const osim* s, double* front, double* ke) {
  double f = -1e300, e = 0.0;
  for (long i = 0; i < s->n; ++i) {
    if (s->x[i][0] > f) f = s->x[i][0];
    e += 0.5 * s->m *
         (s->v[i][0] * s->v[i][0] + s->v[i][1] * s->v[i][1] + s->v[i][2] * s->v[i][2]);
  }
  *front = f;
  *ke = e;
}

static long* user_to_slot(const osim* s) {
  long* slot = (long*)xcalloc((size_t)s->n, sizeof(long));
  for (long k = 0; k < s->n; ++k) slot[s->id[k]] = k;
  return slot;
}

void osph_sample_sigma(const osim* s, long m, const uint32_t* user_ids,
                       double* sigma) {
  long* slot = user_to_slot(s);
  for (long q = 0; q < m; ++q) sigma[q] = sigma_of(s, slot[user_ids[q]]);
  free(slot);
}

/* First acoustic step from rest (v = 0, carried density rate 0, state as set):
 * the step's density summation is evaluated for the sampled particles and
 * all their neighbours, the first half-step leaves positions and densities
 * unchanged and sets p = c0^2 (rho - rho0), and the pressure acceleration of
 * each sampled particle follows (equal to osph_step(1) followed by OSPH_ACC,
 * at the cost of the samples' neighbourhoods only). */
void osph_sample_first_step_acc(const osim* s, long m, const uint32_t* user_ids,
                                double* acc) {
  const double r2max = 4.0 * s->h * s->h;
  long cells[27];
  long* slot = user_to_slot(s);
  char* need = (char*)xcalloc((size_t)s->n, 1);
  double* rho = (double*)xcalloc((size_t)s->n, sizeof(double));
  double* p = (double*)xcalloc((size_t)s->n, sizeof(double));
  for (long q = 0; q < m; ++q) {
    long i = slot[user_ids[q]];
    need[i] = 1;
    int nc = neighbour_cells(s, s->key[i], cells);
    for (int c = 0; c < nc; ++c)
      for (long j = s->cb[cells[c]]; j < s->cb[cells[c] + 1]; ++j)
        if (dist2(s->x[i], s->x[j]) < r2max) need[j] = 1;
  }
  for (long k = 0; k < s->n; ++k)
    if (need[k]) {
      rho[k] = density_of_sigma(s, sigma_of(s, k));
      p[k] = s->c0 * s->c0 * (rho[k] - s->rho0);
    }
  for (long q = 0; q < m; ++q) {
    double a[3];
    pressure_acc_of(s, slot[user_ids[q]], rho, p, a);
    for (int k = 0; k < s->dim; ++k) acc[q * s->dim + k] = a[k];
  }
  free(p);
  free(rho);
  free(need);
  free(slot);
}
