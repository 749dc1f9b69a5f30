// Interaction stages of the weakly-compressible SPH step, templated on the
// dimension D and the pair-arithmetic type T.
//   T = double: FP64 path; records hold absolute positions.
//   T = float : mixed path; records hold float cell-local offsets
//               o = x - (lo + (c + 1/2) s) of the binned cell c, with s the cell
//               edge 2h rounded to float, so a pair distance is o_i - o_j - d s
//               with d the cell offset (-1, 0, 1 per axis) and d s exact in
//               float; state (x, v, rho) stays double.
//
// Direct search (paper, section "Cell linked-list, direct search and
// sorting"): each neighbour loop recomputes kernel values for every particle
// of the 3^D cells around the particle's binned cell; a pair is accepted when
// r^2 < (2h)^2.  Equations (Wendland C2; [Z17] Riemann pressure and density
// relaxation; [Z20] dual time stepping; Adami-style mirrored wall state):
//   density summation  sigma_i = sum_{r<2h} W(r_ij) (fluid + wall, self incl.),
//                      rho_i = rho0 max(sigma_i / sigma0, 1)
//   viscous            a_prior_i = g + (2 mu / rho_i) sum_j V_j (v_i - v_j) W'/(r + 0.01h)
//   half 1             rho += dt/2 drho; p = c0^2 (rho - rho0); x += dt/2 v
//   pressure           a_i = -(2/rho_i) sum_j P*_ij V_j W' e_ij; v += dt (a + a_prior);
//                      x += dt/2 v (first half of the density stage, fused)
//   density            drho_i = -2 rho_i sum_j V_j W' (U_L - U*_ij); rho += dt/2 drho
// with V_j = m / rho_j (walls: V_w = m / rho_w of the mirrored state).
#pragma once

#include <type_traits>

#include "sph_internal.cuh"

namespace sphgb {

namespace stages {

constexpr unsigned kFullMask = 0xffffffffu;

template <int D, class T>
struct Rec;

template <class T>
struct Rec<3, T> {
  using PV = typename Vec4<T>::type;  // (x, y, z, p)
  using SV = typename Vec4<T>::type;  // (vx, vy, vz, rho)
  __device__ static PV makeP(T x, T y, T z, T vx, T vy, T vz, T p) {
    PV r;
    r.x = x; r.y = y; r.z = z; r.w = p;
    return r;
  }
  __device__ static SV makeS(T vx, T vy, T vz, T rho, T p) {
    SV r;
    r.x = vx; r.y = vy; r.z = vz; r.w = rho;
    return r;
  }
  __device__ static T px(const PV& a) { return a.x; }
  __device__ static T py(const PV& a) { return a.y; }
  __device__ static T pz(const PV& a) { return a.z; }
  __device__ static T vx(const PV&, const SV& b) { return b.x; }
  __device__ static T vy(const PV&, const SV& b) { return b.y; }
  __device__ static T vz(const PV&, const SV& b) { return b.z; }
  __device__ static T pres(const PV& a, const SV&) { return a.w; }
  __device__ static T rho(const PV&, const SV& b) { return b.w; }
  __device__ static void set_pos(PV& a, T x, T y, T z) {
    a.x = x; a.y = y; a.z = z;
  }
};

template <class T>
struct Rec<2, T> {
  using PV = typename Vec4<T>::type;  // (x, y, vx, vy)
  using SV = typename Vec2<T>::type;  // (p, rho)
  __device__ static PV makeP(T x, T y, T, T vx, T vy, T, T) {
    PV r;
    r.x = x; r.y = y; r.z = vx; r.w = vy;
    return r;
  }
  __device__ static SV makeS(T, T, T, T rho, T p) {
    SV r;
    r.x = p; r.y = rho;
    return r;
  }
  __device__ static T px(const PV& a) { return a.x; }
  __device__ static T py(const PV& a) { return a.y; }
  __device__ static T pz(const PV&) { return T(0); }
  __device__ static T vx(const PV& a, const SV&) { return a.z; }
  __device__ static T vy(const PV& a, const SV&) { return a.w; }
  __device__ static T vz(const PV&, const SV&) { return T(0); }
  __device__ static T pres(const PV&, const SV& b) { return b.x; }
  __device__ static T rho(const PV&, const SV& b) { return b.y; }
  __device__ static void set_pos(PV& a, T x, T y, T) {
    a.x = x; a.y = y;
  }
};

// Loop records of buffer b.  3D: 8 T per slot, the position record PV in
// T 0-3 and the state record SV in T 4-7, so a neighbour's two records share
// one 32-byte sector in the mixed path and the loops that only read a buffer
// fetch both with one 256-bit gather.  2D: PV (4 T) and SV (2 T) in two
// arrays; a 2D slot padded to 8 T ran 3% slower on batches of small tanks.
template <int D, class T>
struct RecArr {
  using R = Rec<D, T>;
  using PV = typename R::PV;
  using SV = typename R::SV;
  static constexpr int kStride = D == 3 ? 8 : 4;  // T per slot in rec
  T* base;
  SV* sbase;
  __device__ RecArr(const DevBuffers& B, int b)
      : base((T*)B.rec[b]), sbase(D == 3 ? nullptr : (SV*)B.rec_s[b]) {}
  __device__ PV& P(int i) const { return *(PV*)(base + kStride * (size_t)i); }
  __device__ SV& S(int i) const {
    if constexpr (D == 3) return *(SV*)(base + 8 * (size_t)i + 4);
    else return sbase[i];
  }
  // the density slot of S (3D: w, 2D: y)
  __device__ T& rho(int i) const {
    if constexpr (D == 3) return base[8 * (size_t)i + 7];
    else return sbase[i].y;
  }
  // both records of slot j, from a buffer that no thread of the kernel writes
  __device__ void gather(int j, PV& p, SV& s) const {
    if constexpr (D == 3 && std::is_same<T, float>::value) {
      float a[8];
      asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
          : "=f"(a[0]), "=f"(a[1]), "=f"(a[2]), "=f"(a[3]), "=f"(a[4]), "=f"(a[5]),
            "=f"(a[6]), "=f"(a[7])
          : "l"(base + 8 * (size_t)j));
      p = make_float4(a[0], a[1], a[2], a[3]);
      s = make_float4(a[4], a[5], a[6], a[7]);
    } else {
      p = P(j);
      s = S(j);
    }
  }
  // both records of slot i (3D mixed path: one 256-bit store)
  __device__ void store(int i, const PV& p, const SV& s) const {
    if constexpr (D == 3 && std::is_same<T, float>::value) {
      asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                   :: "l"(base + 8 * (size_t)i), "f"(p.x), "f"(p.y), "f"(p.z), "f"(p.w),
                      "f"(s.x), "f"(s.y), "f"(s.z), "f"(s.w)
                   : "memory");
    } else {
      P(i) = p;
      S(i) = s;
    }
  }
};

// wall record: position (absolute or cell-local offset)
template <int D, class T>
struct WallRec;
template <class T>
struct WallRec<3, T> {
  using WV = typename Vec4<T>::type;
  __device__ static WV make(T x, T y, T z) {
    WV r;
    r.x = x; r.y = y; r.z = z; r.w = T(0);
    return r;
  }
  __device__ static T z(const WV& a) { return a.z; }
};
template <class T>
struct WallRec<2, T> {
  using WV = typename Vec2<T>::type;
  __device__ static WV make(T x, T y, T) {
    WV r;
    r.x = x; r.y = y;
    return r;
  }
  __device__ static T z(const WV&) { return T(0); }
};

// constants in the pair type
template <class T>
struct KC {
  T r2max, inv_h, cW, cdW, m, c0, inv_c0, rho0, inv_c0sq, eps, two_mu, cs, half;
  T g[3];
  T riemann;  // 1: Riemann U* in the density relaxation; 0: the average of the states
  // Relaxation loops.  With t = 1 - r / (2h) the kernel slope is
  // W'(r) = cdW (r / h) t^3, so W'(r) e_ij = (cdW / h) t^3 r_ij needs no unit
  // vector; the constant factors of each sum are applied once per particle.
  T neg_inv_2h;  // -1 / (2h): t = 1 + r neg_inv_2h
  T c0_half;     // c0 / 2
  T kP;          // -m cdW / h: a_i = kP / rho_i sum_j 2P*_ij t^3 r_ij / rho_j
  T kD;          // m cdW / h: drho_i = kD rho_i sum_j B_ij t^3 / rho_j
  T kappa2;      // 2 riemann / c0
};

template <class T>
__host__ KC<T> make_kc(const Params& P) {
  KC<T> k;
  k.r2max = (T)P.r2max;
  k.inv_h = (T)(1.0 / P.h);
  k.cW = (T)P.walpha;
  k.cdW = (T)(-5.0 * P.walpha / P.h);
  k.m = (T)P.m;
  k.c0 = (T)P.c0;
  k.inv_c0 = (T)(1.0 / P.c0);
  k.rho0 = (T)P.rho0;
  k.inv_c0sq = (T)(1.0 / P.c0sq);
  k.eps = (T)P.eps;
  k.two_mu = (T)(2.0 * P.mu);
  k.cs = (T)P.cs;
  k.half = (T)0.5;
  k.riemann = (P.variant & kVariantNoRiemann) ? (T)0 : (T)1;
  for (int d = 0; d < 3; ++d) k.g[d] = (T)P.g[d];
  const double cdW_h = -5.0 * P.walpha / (P.h * P.h);
  k.neg_inv_2h = (T)(-0.5 / P.h);
  k.c0_half = (T)(0.5 * P.c0);
  k.kP = (T)(-P.m * cdW_h);
  k.kD = (T)(P.m * cdW_h);
  k.kappa2 = (P.variant & kVariantNoRiemann) ? (T)0 : (T)(2.0 / P.c0);
  return k;
}

// pair-type helpers
// The float forms are the PTX approximations with subnormals flushed: the
// loops never meet a subnormal distance or density, and for normal operands
// they give the same values as rsqrtf / __fdividef without the subnormal
// range handling around them.
__device__ __forceinline__ float inv_sqrt_t(float a) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ double inv_sqrt_t(double a) { return 1.0 / sqrt(a); }
__device__ __forceinline__ float div_t(float a, float b) {
  float r;
  asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ double div_t(double a, double b) { return a / b; }
// a b + c with one rounding, written out where every inlined copy of a loop
// (one-tank and batched kernels, each template choice) must round alike
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// r^2 of the pair: FP64 uses an uncontracted sum (bit-identical acceptance with
// a serial evaluation); float uses ordinary fused arithmetic.
__device__ __forceinline__ double r2_of(double dx, double dy, double dz) {
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}
__device__ __forceinline__ float r2_of(float dx, float dy, float dz) {
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float dsub(float a, float b) { return a - b; }

template <class T>
__device__ __forceinline__ T wendland(const KC<T>& k, T r) {
  T q = r * k.inv_h;
  T t = T(1) - k.half * q;
  T t2 = t * t;
  return k.cW * t2 * t2 * (T(2) * q + T(1));
}
template <class T>
__device__ __forceinline__ T wendland_dr(const KC<T>& k, T r) {
  T q = r * k.inv_h;
  T t = T(1) - k.half * q;
  return k.cdW * q * t * t * t;
}

// Register budget of the neighbour-loop kernels (blocks of up to 256 threads):
// 5 resident blocks -> at most 48 registers in float, 2 -> 128 in double.  The
// 3D density-relaxation loop keeps 4 blocks (64 registers); the one-tank 3D
// pressure loop (k_pressure) measured faster at 5 (1.38 -> 1.33 ms per launch
// on the 5.1 M dam break in storage order, 1.155 -> 1.08 ms in brick order,
// where it spills 16 bytes), the relaxation loop slower (1.12 -> 1.20 ms;
// 0.950 -> 0.977 ms in brick order).
template <class T>
constexpr int kMinBlocks = sizeof(T) == 8 ? 2 : 5;
template <int D, class T>
constexpr int kMinBlocksP = D == 3 && sizeof(T) == 4 ? 4 : kMinBlocks<T>;
template <int D, class T>
constexpr int kMinBlocksPres = D == 3 && sizeof(T) == 4 ? 5 : kMinBlocksP<D, T>;

// Binned cell of a storage slot from its sorted key.
struct Cell {
  int x, y, z;
};
__device__ __forceinline__ Cell decode(uint32_t key, const Params& P) {
  Cell c;
  uint32_t r = key / (uint32_t)P.nx;
  c.x = (int)(key - r * (uint32_t)P.nx);
  c.y = (int)(r % (uint32_t)P.ny);
  c.z = (int)(r / (uint32_t)P.ny);
  return c;
}

// Iterate the 3^D cells around a binned cell in the order dz, dy, dx; f gets
// (cell index, dx, dy, dz).
template <int D, class F>
__device__ __forceinline__ void for_each_cell(const Params& P, Cell c, F&& f) {
  const int kz = D == 3 ? 1 : 0;
  for (int dz = -kz; dz <= kz; ++dz) {
    const int z = c.z + dz;
    if (z < 0 || z >= P.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = c.y + dy;
      if (y < 0 || y >= P.ny) continue;
      const uint32_t row = ((uint32_t)z * (uint32_t)P.ny + (uint32_t)y) * (uint32_t)P.nx;
      for (int dx = -1; dx <= 1; ++dx) {
        const int x = c.x + dx;
        if (x < 0 || x >= P.nx) continue;
        f(row + (uint32_t)x, dx, dy, dz);
      }
    }
  }
}

// Position of a state slot in record form: absolute (FP64) or cell-local offset.
template <class T>
struct Local;
template <>
struct Local<double> {
  static constexpr bool kLocal = false;
  __device__ static void enc(const Params&, const double*, Cell, double x, double y, double z,
                             double& ox, double& oy, double& oz) {
    ox = x; oy = y; oz = z;
  }
};
template <>
struct Local<float> {
  static constexpr bool kLocal = true;
  // Offsets from the cell centre on a pitch that is exact in float, so that
  // o_i - o_j - d * pitch reproduces x_i - x_j without a systematic error from
  // rounding the pitch (the shift d * pitch is then exact in float).
  // centre of cell c along axis k: lo_k + (c + 1/2) pitch (one rounding)
  __device__ static double centre(const Params& P, int k, int c) {
    const double pf = (double)(float)P.cs;
    return __fma_rn((double)c + 0.5, pf, P.lo[k]);
  }
  // ctab, when given, holds the centres of every cell column per axis
  // (nx | ny | nz values, made by centre()): two double operations per axis
  // instead of five on GB300's narrow FP64 pipe
  __device__ static void enc(const Params& P, const double* __restrict__ ctab, Cell c, double x,
                             double y, double z, float& ox, float& oy, float& oz) {
    if (ctab) {
      ox = (float)(x - ctab[c.x]);
      oy = (float)(y - ctab[P.nx + c.y]);
      oz = (float)(z - ctab[P.nx + P.ny + c.z]);
    } else {
      ox = (float)(x - centre(P, 0, c.x));
      oy = (float)(y - centre(P, 1, c.y));
      oz = (float)(z - centre(P, 2, c.z));
    }
  }
};

// ---------------------------------------------------------------------------
// Fixed-point cell-centre offsets (mixed mode, density summation).  A position
// is stored as round((x - centre of its binned cell) * 2^28 / cell edge) in
// int32, so pair differences o_i - o_j - d 2^28 are exact integers and
// r^2 in cell units is the exact integer sum of their squares times 2^-56.
// Offsets are clamped to +-2^29 (only a particle outside the domain, which is
// flagged, can reach that), which keeps every difference within int32.
constexpr int kFxShift = 28;
constexpr long long kFxOne = 1ll << kFxShift;

template <int D>
struct FxRec;
template <>
struct FxRec<3> {
  using V = int4;
};
template <>
struct FxRec<2> {
  using V = int2;
};

__device__ __forceinline__ int fx_of(double x, double centre, double scale) {
  double t = rint((x - centre) * scale);
  t = fmin(fmax(t, -536870912.0), 536870912.0);
  return (int)t;
}

template <int D>
__device__ __forceinline__ typename FxRec<D>::V fx_encode(const Params& P, Cell c, double x,
                                                          double y, double z) {
  const double scale = (double)kFxOne / P.cs;
  typename FxRec<D>::V r;
  r.x = fx_of(x, P.lo[0] + ((double)c.x + 0.5) * P.cs, scale);
  r.y = fx_of(y, P.lo[1] + ((double)c.y + 0.5) * P.cs, scale);
  if constexpr (D == 3) {
    r.z = fx_of(z, P.lo[2] + ((double)c.z + 0.5) * P.cs, scale);
    r.w = 0;
  }
  return r;
}

// Double-float arithmetic on FP32 (value = hi + lo), built from the error-free
// transformations FastTwoSum (Dekker) and TwoProduct with a fused
// multiply-add (Dekker / Ogita-Rump-Oishi); additions carry no multiplications
// other than by powers of two, so no contraction can change them.
struct dfl {
  float hi, lo;
};
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = a + b;
  float e = b - (s - a);
  return {s, e};
}
// a + b for a running sum a with |a.hi| >= |b.hi| (a sum of non-negative
// terms that starts at the largest one): the rounding error of the high
// parts is exact (fast two-sum) and joins the low part, which is
// renormalised once at the end (fast_two_sum(a.hi, a.lo)).
__device__ __forceinline__ dfl df_acc(dfl a, dfl b) {
  const float s = a.hi + b.hi;
  const float e = b.hi - (s - a.hi);
  return {s, a.lo + (e + b.lo)};
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e += a.hi * b.lo + a.lo * b.hi;
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dfl df_sqr(dfl a) {
  float p = a.hi * a.hi;
  float e = fmaf(a.hi, a.hi, -p);
  e += 2.0f * a.hi * a.lo;
  return fast_two_sum(p, e);
}

// Wendland C2 shape (1 - q/2)^4 (2q + 1) = u^4 (5 - 4u), u = 1 - q/2, in
// double-float from the exact integer r^2 in fixed-point units (R2 = r^2 2^56
// / cell^2; the cell edge is 2h, so q = 2 sqrt(R2) 2^-28 = sqrt(R2) 2^-27),
// for R2 < 2^56.  R2 splits into 23-bit limbs l0 + l1 2^23 + l2 2^46, each
// turned into an exact float by placing it in the mantissa of a power of two
// (2^23, 2^46, 2^69) and subtracting that power (no integer-to-float
// conversion: the 64-bit ones measured slow enough to bound the kernel); two
// fast two-sums give hi + lo = R2 to about 2^-48.  s = hi y with y the
// approximate reciprocal square root (relative error about 2^-22), and one
// Newton step s + (R2 - s^2) y / 2 leaves a relative error near 2^-43 in the
// root (R2 = 0, coincident particles: y = 1, s = 0, q = 0).  With 0 <= q <= 2
// both 1 - q/2 and 5 - 4u are exact fast two-sums.
__device__ __forceinline__ dfl wendland_shape_fx(unsigned long long R2) {
  const uint32_t w0 = (uint32_t)R2, w1 = (uint32_t)(R2 >> 32);
  const uint32_t l0 = w0 & 0x7FFFFFu;
  const uint32_t l1 = __funnelshift_r(w0, w1, 23) & 0x7FFFFFu;
  const uint32_t l2 = w1 >> 14;
  const float f0 = __uint_as_float(0x4B000000u | l0) - 0x1p23f;  // l0
  const float f1 = __uint_as_float(0x56800000u | l1) - 0x1p46f;  // l1 2^23
  const float f2 = __uint_as_float(0x62000000u | l2) - 0x1p69f;  // l2 2^46
  // exact: f2 is 0 or >= 2^46 > f1, and the partial sum 0 or >= 2^23 > f0
  const dfl a = fast_two_sum(f2, f1);
  const dfl b = fast_two_sum(a.hi, f0);
  const float hi = b.hi;
  const float lo = b.lo + a.lo;
  const float y = inv_sqrt_t(fmaxf(hi, 1.0f));
  const float s = hi * y;
  const float e = fmaf(s, s, -hi);  // s^2 - hi
  const float s_lo = (lo - e) * (0.5f * y);
  const float qh = s * 0x1p-27f, ql = s_lo * 0x1p-27f;
  dfl u = fast_two_sum(1.0f, -0.5f * qh);
  u.lo -= 0.5f * ql;
  u = fast_two_sum(u.hi, u.lo);
  const dfl u4 = df_sqr(df_sqr(u));
  dfl v = fast_two_sum(5.0f, -4.0f * u.hi);
  v.lo -= 4.0f * u.lo;
  v = fast_two_sum(v.hi, v.lo);
  return df_mul(u4, v);
}

// Pointers of one state copy, chosen with selects (runtime indexing into the
// kernel-parameter arrays would force them into local memory).
template <class T>
struct Live {
  double *x0, *x1, *x2, *v0, *v1, *v2, *rho;
  T* drho;
  uint32_t* id;
};
template <class T>
__device__ __forceinline__ Live<T> live(const DevBuffers& B, int par) {
  Live<T> L;
  L.x0 = par ? B.x[1][0] : B.x[0][0];
  L.x1 = par ? B.x[1][1] : B.x[0][1];
  L.x2 = par ? B.x[1][2] : B.x[0][2];
  L.v0 = par ? B.v[1][0] : B.v[0][0];
  L.v1 = par ? B.v[1][1] : B.v[0][1];
  L.v2 = par ? B.v[1][2] : B.v[0][2];
  L.rho = par ? B.rho[1] : B.rho[0];
  L.drho = (T*)(par ? B.drho[1] : B.drho[0]);
  L.id = par ? B.id[1] : B.id[0];
  return L;
}

__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFullMask, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// Reorder after the sort: gather slot j of the live state copy into slot k of
// the other copy and write the loop records of buffer 0 (positions; velocity;
// old p; old rho) for binned cell key `key` (in the tank's grid).
// Drift budget of a particle for the lists of the advection step that
// begins: its own speed (plus what gravity adds) over the step and one
// overshooting acoustic step, with margin, and a floor; at most bmax (half
// the step's skin).  Any value is valid (the lists and the checks use the
// same one); this one is sized so that it is rarely left.
__device__ __forceinline__ float drift_budget(float speed, float gspan, float span, float floor_,
                                             float bmax) {
  const float b = 1.25f * (speed + gspan) * span + floor_;
  return b < bmax ? b : bmax;
}

// Budget constants of an advection step, computed once per launch or tile.
struct BudgetArgs {
  float span, gspan, floor_, bmax;
};
__device__ __forceinline__ BudgetArgs budget_args(const Params& P, const DevScalars& sc) {
  const double span = sc.dt_ad + 1.5 * sc.dt_ac;
  const double g = sqrt(P.g[0] * P.g[0] + P.g[1] * P.g[1] + P.g[2] * P.g[2]);
  return BudgetArgs{(float)span, (float)(g * span), (float)(0.01 * P.h), (float)(0.5 * sc.skin)};
}

// Build record of a slot: record-frame position and drift budget.
template <int D, class T>
__device__ __forceinline__ typename Vec4<T>::type build_rec(T ox, T oy, T oz, T b) {
  typename Vec4<T>::type r;
  r.x = ox; r.y = oy; r.z = D == 3 ? oz : T(0); r.w = b;
  return r;
}

template <int D, class T>
__device__ __forceinline__ void reorder_slot(const Params& P, const DevBuffers& B,
                                             const Live<T>& S, const Live<T>& Dd, int k,
                                             uint32_t j, uint32_t key, const BudgetArgs& ba) {
  using R = Rec<D, T>;
  const RecArr<D, T> rec(B, 0);
  if (!SPH_DBG_IN(B, j, P.foff, P.foff + P.n)) return;
  {
    double x = S.x0[j], y = S.x1[j], z = D == 3 ? S.x2[j] : 0.0;
    double vx = S.v0[j], vy = S.v1[j], vz = D == 3 ? S.v2[j] : 0.0;
    double rho = S.rho[j];
    Dd.x0[k] = x;
    Dd.x1[k] = y;
    Dd.v0[k] = vx;
    Dd.v1[k] = vy;
    if (D == 3) {
      Dd.x2[k] = z;
      Dd.v2[k] = vz;
    }
    Dd.rho[k] = rho;
    Dd.drho[k] = S.drho[j];
    Dd.id[k] = S.id[j];
    const float fvx = (float)vx, fvy = (float)vy, fvz = (float)vz;
    const float bk = drift_budget(sqrtf(fvx * fvx + fvy * fvy + fvz * fvz), ba.gspan, ba.span,
                                  ba.floor_, ba.bmax);
    B.bud[k] = bk;
    T ox, oy, oz;
    const Cell ck = decode(key, P);
    Local<T>::enc(P, B.ctab, ck, x, y, z, ox, oy, oz);
    ((T*)B.xreb[0])[k] = ox;
    ((T*)B.xreb[1])[k] = oy;
    if (D == 3) ((T*)B.xreb[2])[k] = oz;
    ((typename Vec4<T>::type*)B.brec)[k] = build_rec<D, T>(ox, oy, oz, (T)bk);
    T p = (T)(P.c0sq * (rho - P.rho0));
    rec.store(k, R::makeP(ox, oy, oz, (T)vx, (T)vy, (T)vz, p),
              R::makeS((T)vx, (T)vy, (T)vz, (T)rho, p));
    if constexpr (Local<T>::kLocal)
      ((typename FxRec<D>::V*)B.recI)[k] = fx_encode<D>(P, ck, x, y, z);
  }
}

// Loop records of buffer 0 from the live state as it stands (no update), in
// the frame of each slot's binned cell: the positions a list build reads.
template <int D, class T>
__global__ void k_encode_records(Params P, DevBuffers B) {
  using R = Rec<D, T>;
  const Live<T> S = live<T>(B, B.sc->par);
  const RecArr<D, T> rec(B, 0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    const double x = S.x0[i], y = S.x1[i], z = D == 3 ? S.x2[i] : 0.0;
    const double vx = S.v0[i], vy = S.v1[i], vz = D == 3 ? S.v2[i] : 0.0;
    const double rho = S.rho[i];
    T ox, oy, oz;
    Local<T>::enc(P, B.ctab, decode(B.binned[i], P), x, y, z, ox, oy, oz);
    const T p = (T)(P.c0sq * (rho - P.rho0));
    rec.store(i, R::makeP(ox, oy, oz, (T)vx, (T)vy, (T)vz, p),
              R::makeS((T)vx, (T)vy, (T)vz, (T)rho, p));
  }
}

template <int D, class T>
__global__ void k_reorder(Params P, DevBuffers B, int gated) {
  DevScalars* sc = B.sc;
  if (gated && !sc->new_adv) return;
  const int par = sc->par;
  const Live<T> S = live<T>(B, par), Dd = live<T>(B, par ^ 1);
  const uint32_t* __restrict__ perm = B.vals[B.sorted_buf];
  const uint32_t* __restrict__ keys = B.keys[B.sorted_buf];
  const BudgetArgs ba = budget_args(P, *sc);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.n; k += gridDim.x * blockDim.x)
    reorder_slot<D, T>(P, B, S, Dd, k, perm[k], keys[k], ba);
}

// ---------------------------------------------------------------------------
// Processing order of the one-tank 3D mixed neighbour loops (list build,
// density summation, viscous force, pressure and density relaxation; the
// neighbour-search benchmark's density pass too), made at every rebuild: the
// 32-slot groups (a warp's slots and list block) sorted by the brick of
// 2^kBrickLog2 cells per axis (4 x 4 x 4) that holds each group's first slot.
// The warps of one multiprocessor then walk neighbouring bricks together, so
// the records they gather stay in its L1 longer than along the cell rows of
// the storage order.  The order of the groups within a brick is left to the
// atomics: the loops give the same results in any order.
__device__ __forceinline__ uint32_t brick_of(const Cell& c, const Params& P) {
  const int nbx = (P.nx + (1 << kBrickLog2X) - 1) >> kBrickLog2X;
  const int nby = (P.ny + (1 << kBrickLog2Y) - 1) >> kBrickLog2Y;
  return (uint32_t)((c.x >> kBrickLog2X) +
                    nbx * ((c.y >> kBrickLog2Y) + nby * (c.z >> kBrickLog2Z)));
}

// (also zeroes the claim counters of the rebuild's loops: list build,
// density summation, viscous force)
template <int D>
__global__ void k_units_clear(Params P, DevBuffers B, int gated) {
  if (gated && !B.sc->new_adv) return;
  const uint32_t nb = brick_count(P);
  const uint32_t nc = 3u * (uint32_t)B.parts;
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b <= nb || b < nc;
       b += gridDim.x * blockDim.x) {
    if (b <= nb) B.brick_start[b] = 0;
    if (b < nb) B.brick_fill[b] = 0;
    if (b < nc) B.unit_ctr[2 * B.parts + b] = 0;
  }
}

template <int D>
__global__ void k_units_count(Params P, DevBuffers B, int gated) {
  if (gated && !B.sc->new_adv) return;
  const int ng = (P.n + 31) >> 5;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
    const uint32_t b = brick_of(decode(B.binned[g * 32], P), P);
    B.unit_brick[g] = b;
    atomicAdd(&B.brick_start[b], 1u);
  }
}

// exclusive scan of the brick counts in place (one block of kUnitScanThreads)
constexpr int kUnitScanThreads = 1024;
template <int D>
__global__ void __launch_bounds__(kUnitScanThreads) k_units_scan(Params P, DevBuffers B,
                                                                 int gated) {
  if (gated && !B.sc->new_adv) return;
  __shared__ uint32_t part[kUnitScanThreads / 32];
  const uint32_t nb = brick_count(P);
  const uint32_t chunk = (nb + kUnitScanThreads - 1) / kUnitScanThreads;
  const uint32_t b0 = threadIdx.x * chunk;
  const uint32_t b1 = min(b0 + chunk, nb);
  uint32_t local = 0;
  for (uint32_t b = b0; b < b1; ++b) local += B.brick_start[b];
  // block-wide exclusive scan of the per-thread sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = local;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(kFullMask, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) part[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = part[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(kFullMask, w, o);
      if (lane >= o) w += v;
    }
    part[lane] = w;
  }
  __syncthreads();
  uint32_t run = incl - local + (warp > 0 ? part[warp - 1] : 0u);
  for (uint32_t b = b0; b < b1; ++b) {
    const uint32_t c = B.brick_start[b];
    B.brick_start[b] = run;
    run += c;
  }
  if (threadIdx.x == kUnitScanThreads - 1) B.brick_start[nb] = run;
}

template <int D>
__global__ void k_units_scatter(Params P, DevBuffers B, int gated) {
  if (gated && !B.sc->new_adv) return;
  const int ng = (P.n + 31) >> 5;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
    const uint32_t b = B.unit_brick[g];
    B.units[B.brick_start[b] + atomicAdd(&B.brick_fill[b], 1u)] = (uint32_t)g;
  }
}

// ---------------------------------------------------------------------------
// Slots one thread of a loop body visits: i, i + stride, ... < end.
struct StrideSlots {
  int i, end, stride;
  template <class F>
  __device__ __forceinline__ void each(F&& f) const {
    for (int k = i; k < end; k += stride) f(k);
  }
};

__device__ __forceinline__ int sm_id() {
  int r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

// Slots of the groups in brick order (DevBuffers::units): the order is cut
// into `parts` runs of near-equal length; a warp claims one group at a time
// (lane 0, one atomic) from the run of its multiprocessor, and when that is
// done looks for any run with groups left (its lanes test 32 runs per load),
// so every group is processed once whatever the multiprocessor numbering.
// ctr holds the runs' claim counters (zeroed before the launch).
struct UnitSlots {
  const uint32_t* units;
  uint32_t* ctr;
  int parts, ngroups, end;
  template <class F>
  __device__ __forceinline__ void each(F&& f) const {
    const int lane = threadIdx.x & 31;
    const int base = ngroups / parts, rem = ngroups - base * parts;
    int p = sm_id() % parts;
    for (;;) {
      const int u0 = p * base + min(p, rem);
      const int size = base + (p < rem ? 1 : 0);
      for (;;) {
        int u = size;
        if (lane == 0 && *(volatile uint32_t*)(ctr + p) < (uint32_t)size)
          u = (int)atomicAdd(ctr + p, 1u);
        u = __shfl_sync(kFullMask, u, 0);
        if (u >= size) break;
        const uint32_t g = units[u0 + u];
        const int i = (int)(g * 32u) + lane;
        if (g < (uint32_t)ngroups && i < end) f(i);
      }
      // another run with unclaimed groups, if any
      int next = -1;
      for (int r = 0; r < parts - 1 && next < 0; r += 32) {
        int q = p + 1 + r + lane;
        if (q >= parts) q -= parts;
        const bool open = r + lane < parts - 1 &&
                          *(volatile uint32_t*)(ctr + q) < (uint32_t)(base + (q < rem ? 1 : 0));
        const unsigned m = __ballot_sync(kFullMask, open);
        if (m) next = __shfl_sync(kFullMask, q, __ffs(m) - 1);
      }
      if (next < 0) return;
      p = next;
    }
  }
};

// ---------------------------------------------------------------------------
// Neighbour lists.  Direct search tests every particle of the 3^D cells
// (about 475 in 3D) for about 81 accepted neighbours, and the pair arithmetic
// then runs with few lanes of a warp active.  Right after each rebuild every
// particle i records the candidates j closer than 2h + b_i + b_j, in
// candidate order (fluid particles by cells dz, dy, dx, then wall particles
// in the same cell order); the other loops of the advection step walk that list instead of the
// cells.  b_k is particle k's drift budget, set by the reorder from its own
// speed (walls: the translating walls' speed bound, 0 at rest).
//
// Exactness: a candidate left out was at least 2h + b_i + b_j away at the
// rebuild; while neither particle has moved more than its budget since then,
// it is still farther than 2h, so the accepted set -- and, since the list
// keeps candidate order, every sum -- is the same as with direct search.
// The kernels that move particles (first half-step, pressure kick and drift,
// transport shift) test every particle against its budget at the positions
// the next loop reads and set a flag for that loop (drift_bad_p: pressure
// and, at the rebuild, viscous; drift_bad_r: density relaxation); a loop uses
// the list only while its flag is clear and no list overflowed, and falls
// back to direct search otherwise, until the next rebuild.  A budget follows
// the particle's own speed rather than the fastest particle's, so the lists
// carry few more entries than the pairs within 2h.
//
// Entry: neighbour index in bits 0..25 and (dx + 1) | (dy + 1) << 2 |
// (dz + 1) << 4 in bits 26..31 (particle and wall counts below 2^26).  A list
// holds the fluid neighbours first and the wall neighbours after them, so a
// loop walks two runs of one kind each instead of testing a flag per entry;
// nl_cnt packs the two run lengths (fluid in bits 0..15, wall in bits 16..31).
// Entry k of particle i lives at ((i / 32) cap + k) 32 + i % 32, so a warp's
// k-th entries are one coalesced 128-byte line.
constexpr int kIdxBits = 26;
constexpr uint32_t kIdxMask = (1u << kIdxBits) - 1u;

__device__ __forceinline__ uint32_t nl_code(int dx, int dy, int dz) {
  return (uint32_t)((dx + 1) | ((dy + 1) << 2) | ((dz + 1) << 4)) << kIdxBits;
}
__device__ __forceinline__ size_t nl_slot(int i, int k, int cap) {
  return ((size_t)(i >> 5) * (size_t)cap + (size_t)k) * 32u + (size_t)(i & 31);
}

// Appends the entries of one particle in visiting order (every fluid
// candidate before any wall candidate); counts past the capacity are kept so
// the caller can flag the overflow.
struct ListWriter {
  uint32_t* nl;
  int cap, i, nf, nw;
  __device__ __forceinline__ void add(uint32_t entry, bool w) {
    const int k = nf + nw;
    if (k < cap) nl[nl_slot(i, k, cap)] = entry;
    if (w) ++nw; else ++nf;
  }
  __device__ __forceinline__ bool overflowed() const { return nf + nw > cap; }
  __device__ __forceinline__ uint32_t packed() const {
    const int f = min(nf, cap);
    return (uint32_t)f | ((uint32_t)min(nw, cap - f) << 16);
  }
};

// The cell offsets of a list entry as floats: bits 26..31 of an entry hold
// (dx + 1) | (dy + 1) << 2 | (dz + 1) << 4, so the float loops read
// (dx, dy, dz) from this 64-entry table in shared memory (one load) instead
// of decoding and converting three fields.  Every block fills it once.
struct ShiftTable {
  float4 d[64];
};
__device__ __forceinline__ void fill_shift_table(ShiftTable& t) {
  for (int c = threadIdx.x; c < 64; c += blockDim.x)
    t.d[c] = make_float4((float)((c & 3) - 1), (float)(((c >> 2) & 3) - 1),
                         (float)(((c >> 4) & 3) - 1), 0.0f);
  __syncthreads();
}

// The float c - 1 of a shift code c in {0, 1, 2} without a table or a
// conversion: its two high bytes (0xBF80, 0x0000, 0x3F80) picked out of two
// constants by one byte permute.
__device__ __forceinline__ float shift_f(uint32_t c) {
  return __uint_as_float(__byte_perm(0x003F00BFu, 0x00800080u, c * 0x1100u + 0x0433u));
}

// Which float loops take the shifts from the entry bits (shift_f) rather than
// the shared-memory table: measured per loop on the 5.1 M 3D dam break and the
// 256 2D tanks (same values either way), every 3D loop ran faster without the
// table's shared-memory reads (pressure 1.62 -> 1.44 ms per launch), every 2D
// loop slower.
template <int D>
constexpr bool kShiftBits = D == 3;

// The last argument of a visitor call says whether the candidate may be the
// target itself: direct search meets i in its own cell, a list never holds it
// (a compile-time constant, so the list walks carry no self test).
using MaySelf = std::true_type;
using NotSelf = std::false_type;
constexpr NotSelf kNotSelf{};
constexpr MaySelf kMaySelf{};

// One run of list entries [k0, k1) of one kind; entries are prefetched two
// ahead, so the list streams from DRAM while the previous pairs are computed.
// The walk is unrolled by two, which lets the compiler issue the next pair's
// record gathers before this pair's arithmetic (same order of the sums;
// measured +1.5% on the 5.1 M 3D dam break, +0.6% on the 256 2D tanks).
template <bool kTab, bool kBits, bool kWall, class V>
__device__ __forceinline__ void walk_list(const Params& P, const DevBuffers& B,
                                          const uint32_t* __restrict__ e, int k0, int k1, V& v,
                                          const ShiftTable* tab) {
  uint32_t x0 = k0 < k1 ? __ldcs(e + (size_t)k0 * 32u) : 0u;
  uint32_t x1 = k0 + 1 < k1 ? __ldcs(e + (size_t)(k0 + 1) * 32u) : 0u;
#pragma unroll 2
  for (int k = k0; k < k1; ++k) {
    const uint32_t x = x0;
    x0 = x1;
    x1 = k + 2 < k1 ? __ldcs(e + (size_t)(k + 2) * 32u) : 0u;
    const int j = (int)(x & kIdxMask);
    if (!SPH_DBG_IN(B, j, kWall ? P.woff : P.foff, kWall ? P.woff + P.nw : P.foff + P.n))
      continue;
    if constexpr (kBits) {
      const uint32_t c = x >> kIdxBits;
      v(j, shift_f(c & 3u), shift_f((c >> 2) & 3u), shift_f(c >> 4), kWall, kNotSelf);
    } else if constexpr (kTab) {
      const float4 d = tab->d[x >> kIdxBits];
      v(j, d.x, d.y, d.z, kWall, kNotSelf);
    } else {
      const uint32_t c = x >> kIdxBits;
      v(j, (int)(c & 3u) - 1, (int)((c >> 2) & 3u) - 1, (int)(c >> 4) - 1, kWall, kNotSelf);
    }
  }
}

// Rows 0 .. n-1 of the list block of a group of 32 slots (128 bytes a row,
// group base `g`), n the longest list of the warp's active lanes, fetched into
// L2 with one bulk prefetch issued by the lowest active lane before the walk:
// the walk's row loads then wait for L2 rather than DRAM.  A hint only (no
// completion to wait for); the rows lie inside the group's list_cap rows.
__device__ __forceinline__ void prefetch_list_rows(const uint32_t* g, int n) {
  const unsigned am = __activemask();
  const int mx = __reduce_max_sync(am, n);
  if ((int)(threadIdx.x & 31) == __ffs(am) - 1 && mx > 0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(g), "r"(mx * 128)
                 : "memory");
}

// Visit the candidates of target i either through its list or through the
// 3^D cells: every fluid candidate (cells dz, dy, dx; ascending index), then
// every wall candidate in the same cell order.  v(j, dx, dy, dz, wall) does
// the test and the arithmetic; the wall argument is a constant at each call
// site.  With kTab the list path passes the offsets as floats from `tab`, with
// kBits as floats from shift_f (the same values; direct search passes ints).
template <int D, bool kTab = false, bool kBits = false, class V>
__device__ __forceinline__ void visit_neighbours(const Params& P, const DevBuffers& B, Cell ci,
                                                 int i, bool use_list, V&& v,
                                                 const ShiftTable* tab = nullptr) {
  if (!SPH_DBG_IN(B, ci.x, 0, P.nx) || !SPH_DBG_IN(B, ci.y, 0, P.ny) ||
      !SPH_DBG_IN(B, ci.z, 0, D == 3 ? P.nz : 1))
    return;
  if (use_list) {
    const uint32_t c = B.nl_cnt[i];
    const int nf = (int)(c & 0xFFFFu);
    const int nt = nf + (int)(c >> 16);
    const uint32_t* __restrict__ e = B.nl + nl_slot(i, 0, P.list_cap);
    prefetch_list_rows(e - (i & 31), nt);
    walk_list<kTab, kBits, false>(P, B, e, 0, nf, v, tab);
    walk_list<kTab, kBits, true>(P, B, e, nf, nt, v, tab);
    return;
  }
  const uint32_t* __restrict__ cb = B.cell_begin + P.cell_base;
  for_each_cell<D>(P, ci, [&](uint32_t c, int dx, int dy, int dz) {
    const uint32_t e = cb[c + 1];
    if (SPH_DBG_IN(B, cb[c], P.foff, P.foff + P.n + 1) &&
        SPH_DBG_IN(B, e, cb[c], P.foff + P.n + 1))
      for (uint32_t j = cb[c]; j < e; ++j) v((int)j, dx, dy, dz, false, kMaySelf);
  });
  if (P.nw > 0) {
    const uint32_t* __restrict__ wcb = B.wall_cb + P.cell_base;
    for_each_cell<D>(P, ci, [&](uint32_t c, int dx, int dy, int dz) {
      const uint32_t we = wcb[c + 1];
      if (SPH_DBG_IN(B, wcb[c], P.woff, P.woff + P.nw + 1) &&
          SPH_DBG_IN(B, we, wcb[c], P.woff + P.nw + 1))
        for (uint32_t w = wcb[c]; w < we; ++w) v((int)w, dx, dy, dz, true, kNotSelf);
    });
  }
}

// x - d * cs in the record frame (x itself for absolute positions); d is the
// cell offset, an int or the same value as a float (ShiftTable)
template <class T>
__device__ __forceinline__ T shifted(T x, int d, T cs) {
  if constexpr (!Local<T>::kLocal) return x;
  return fmaf(-(float)d, cs, x);
}
template <class T>
__device__ __forceinline__ T shifted(T x, float d, T cs) {
  if constexpr (!Local<T>::kLocal) return x;
  return fmaf(-d, cs, x);
}

// Whether this launch may use the lists: no list overflowed, no particle has
// left its drift budget at the positions the loop reads (drift_bad: the flag
// for those positions), and the translating walls, at the loop's time
// t_eval, are within theirs.
__device__ __forceinline__ bool list_ok(const Params& P, const DevScalars* sc, int drift_bad,
                                        double t_eval) {
  return P.use_list && !sc->list_bad && !drift_bad &&
         P.wall_vmax * (t_eval - sc->t_reb) <= sc->wall_budget;
}

// Whether particle i, at record-frame position (ox, oy, oz) (relative to the
// cell it was binned in, as at the rebuild), has moved farther than its
// budget since the rebuild.  In float the offsets carry errors of a few
// 1e-7 of a cell edge, far below the budgets' floor of 0.01 h, so the test
// at 0.999 b is conservative; flag_drift records it block-wide.
template <int D, class T>
__device__ __forceinline__ bool drifted(const DevBuffers& B, int i, T ox, T oy, T oz) {
  const T dx = ox - ((const T*)B.xreb[0])[i], dy = oy - ((const T*)B.xreb[1])[i];
  const T dz = D == 3 ? oz - ((const T*)B.xreb[2])[i] : T(0);
  const T b = T(0.999) * (T)B.bud[i];
  return dx * dx + dy * dy + dz * dz > b * b;
}
// (a warp vote, no block barrier: the batched kernels call the bodies once
// per tile; the atomic runs only where a particle has drifted out)
__device__ __forceinline__ void flag_drift(int* flag, int any) {
  if (__any_sync(kFullMask, any) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

// Pair geometry shared by the loops: r_ij = x_i - x_j of neighbour j.
template <int D, class T>
struct PairGeo {
  using R = Rec<D, T>;
  using WR = WallRec<D, T>;
  RecArr<D, T> rec;
  const typename WR::WV* __restrict__ wall;
  T xi, yi, zi;
  T cs;
  template <class S>
  __device__ __forceinline__ void rel_rec(const typename R::PV& pj, S dx, S dy, S dz, T& rx,
                                          T& ry, T& rz) const {
    rx = dsub(shifted<T>(xi, dx, cs), R::px(pj));
    ry = dsub(shifted<T>(yi, dy, cs), R::py(pj));
    rz = dsub(shifted<T>(zi, dz, cs), R::pz(pj));
  }
  template <class S>
  __device__ __forceinline__ void rel_wall(const typename WR::WV& pw, S dx, S dy, S dz, T& rx,
                                           T& ry, T& rz) const {
    rx = dsub(shifted<T>(xi, dx, cs), pw.x);
    ry = dsub(shifted<T>(yi, dy, cs), pw.y);
    rz = dsub(shifted<T>(zi, dz, cs), WR::z(pw));
  }
  template <class S>
  __device__ __forceinline__ void rel(int j, S dx, S dy, S dz, bool w, T& rx, T& ry,
                                      T& rz) const {
    const T bx = shifted<T>(xi, dx, cs);
    const T by = shifted<T>(yi, dy, cs);
    const T bz = shifted<T>(zi, dz, cs);
    if (w) {
      const typename WR::WV pw = wall[j];
      rx = dsub(bx, pw.x); ry = dsub(by, pw.y); rz = dsub(bz, WR::z(pw));
    } else {
      const typename R::PV pj = rec.P(j);
      rx = dsub(bx, R::px(pj)); ry = dsub(by, R::py(pj)); rz = dsub(bz, R::pz(pj));
    }
  }
};

// v_w . e for wall particle j with a prescribed velocity (kVariantMovingWall):
// a wall sliding along itself keeps its position; its velocity enters the
// mirrored state v_R = 2 v_w - v_i, so U_R = -U_L - 2 v_w . e.
template <int D, class T>
__device__ __forceinline__ T wall_vel_dot(const DevBuffers& B, int j, T ex, T ey, T ez) {
  using WR = WallRec<D, T>;
  const typename WR::WV vw = ((const typename WR::WV*)B.wall_vel)[j];
  return vw.x * ex + vw.y * ey + WR::z(vw) * ez;
}

// (x_i - x_w) . a_w for an oscillating wall particle j (kVariantAccelWall):
// with it the mirrored wall pressure p_w = p_i + rho_i (x_w - x_i).(g - a_w).
template <int D, class T>
__device__ __forceinline__ T wall_acc_dot(const DevBuffers& B, int j, T rx, T ry, T rz) {
  using WR = WallRec<D, T>;
  const typename WR::WV aw = ((const typename WR::WV*)B.wall_acc)[j];
  return aw.x * rx + aw.y * ry + WR::z(aw) * rz;
}

// List build (right after the rebuild, positions = binned positions): one
// direct search per particle that records the candidates closer than
// 2h + skin.  The membership test runs in the pair type on the build records;
// its rounding is far below the skin, so the list is a superset of every
// pair the later loops accept.
//
// Every loop below is a body over the slots i, i + stride, ... < end of one
// tank (the whole fluid for one tank; one tile of a batch), ending with the
// block-wide reductions; k_* are the one-tank kernels around them.
// A candidate j enters i's list when closer than 2h + b_i + b_j (b the drift
// budgets of the rebuild, or larger ones when lists are restored): while no
// particle leaves its budget, a pair left out stays farther than 2h.  Each
// candidate is one 16-byte gather of its build record (position, budget).
template <int D, class T, class Slots>
__device__ __forceinline__ void build_lists_slots(const Params& P, const DevBuffers& B,
                                                  const KC<T>& k, DevScalars* sc,
                                                  const Slots& slots) {
  using R = Rec<D, T>;
  using BV = typename Vec4<T>::type;
  const BV* __restrict__ brec = (const BV*)B.brec;
  const RecArr<D, T> rec(B, 0);
  const uint32_t* __restrict__ keys = B.binned;
  const T two_h = (T)(2.0 * P.h);
  const T bw = (T)sc->wall_budget;
  const T grow = (T)(1.0 + 1e-6);
  int overflow = 0;
  slots.each([&](const int i) {
    const Cell ci = decode(keys[i], P);
    const BV pi = brec[i];
    PairGeo<D, T> G{rec, (const typename WallRec<D, T>::WV*)B.wallP, pi.x, pi.y, pi.z, k.cs};
    ListWriter L{B.nl, P.list_cap, i, 0, 0};
    const T ri = two_h + pi.w;
    visit_neighbours<D>(P, B, ci, i, false, [&](int j, int dx, int dy, int dz, bool w, auto) {
      T rx, ry, rz, bj;
      if (w) {
        G.rel_wall(G.wall[j], dx, dy, dz, rx, ry, rz);
        bj = bw;
      } else {
        const BV pj = brec[j];
        rx = dsub(shifted<T>(G.xi, dx, G.cs), pj.x);
        ry = dsub(shifted<T>(G.yi, dy, G.cs), pj.y);
        rz = dsub(shifted<T>(G.zi, dz, G.cs), pj.z);
        bj = pj.w;
      }
      const T rl = (ri + bj) * grow;
      if (r2_of(rx, ry, rz) < rl * rl && (w || j != i))
        L.add((uint32_t)j | nl_code(dx, dy, dz), w);
    });
    B.nl_cnt[i] = L.packed();
    if (L.overflowed()) overflow = 1;
  });
  if (__syncthreads_or(overflow) && threadIdx.x == 0) atomicOr(&sc->list_bad, 1);
}

template <int D, class T>
__device__ __forceinline__ void build_lists_range(const Params& P, const DevBuffers& B,
                                                  const KC<T>& k, DevScalars* sc, int i, int end,
                                                  int stride) {
  build_lists_slots<D, T>(P, B, k, sc, StrideSlots{i, end, stride});
}

// kUnits: the slots in brick order (one tank, 3D mixed), else strided.
template <int D, class T, bool kUnits = false>
__global__ void __launch_bounds__(256, kMinBlocks<T>) k_build_lists(Params P, DevBuffers B, KC<T> k,
                                                                    int gated) {
  DevScalars* sc = B.sc;
  if (!P.use_list || (gated && !sc->new_adv)) return;
  if constexpr (kUnits)
    build_lists_slots<D, T>(
        P, B, k, sc, UnitSlots{B.units, B.unit_ctr + 2 * B.parts, B.parts, (P.n + 31) >> 5, P.n});
  else
    build_lists_range<D, T>(P, B, k, sc, blockIdx.x * blockDim.x + threadIdx.x, P.n,
                            gridDim.x * blockDim.x);
}

// Density from the kernel sum: the free-surface clamp rho0 max(sigma/sigma0, 1),
// or the blended reinitialisation rho_sum + max(0, rho_prev - rho_sum) rho0 /
// rho_prev with rho_sum = rho0 sigma / sigma0 and rho_prev the density carried
// into the summation.
__device__ __forceinline__ double reinit_density(const Params& P, double sigma, double rho_prev) {
  const double ratio = sigma / P.sigma0;
  if (!(P.variant & kVariantBlended)) return P.rho0 * (ratio > 1.0 ? ratio : 1.0);
  const double rho_sum = P.rho0 * ratio;
  const double excess = rho_prev - rho_sum;
  return rho_sum + (excess > 0.0 ? excess : 0.0) * P.rho0 / rho_prev;
}

// Density summation (FP64 path): reads records P of buffer 0; writes rho
// (state) and the rho slot of records S of buffer 0.  Self is part of the
// sum (W(0)) and comes first; direct search skips i where it meets it (a list
// never holds it), so both visit the other particles in the same order.
template <int D, class T>
__device__ __forceinline__ void density_summation_range(const Params& P, const DevBuffers& B,
                                                        const KC<T>& k, DevScalars* sc, int i,
                                                        int end, int stride) {
  using R = Rec<D, T>;
  const bool use_list = list_ok(P, sc, sc->drift_bad_p, sc->t_reb);
  double* rho_live = sc->par ? B.rho[1] : B.rho[0];
  const RecArr<D, T> rec(B, 0);
  const uint32_t* __restrict__ keys = B.binned;
  for (; i < end; i += stride) {
    const Cell ci = decode(keys[i], P);
    const typename R::PV pi = rec.P(i);
    PairGeo<D, T> G{rec, (const typename WallRec<D, T>::WV*)B.wallP, R::px(pi), R::py(pi),
                    R::pz(pi), k.cs};
    T sig = wendland(k, T(0));
    visit_neighbours<D>(P, B, ci, i, use_list,
                        [&](int j, int dx, int dy, int dz, bool w, auto may_self) {
      if (may_self && !w && j == i) return;
      T rx, ry, rz;
      G.rel(j, dx, dy, dz, w, rx, ry, rz);
      const T r2 = r2_of(rx, ry, rz);
      if (r2 < k.r2max) sig += wendland(k, sqrt(r2));
    });
    const double rho = reinit_density(P, (double)sig, rho_live[i]);
    if (P.variant & kVariantTransport) B.sigma64[i] = (double)sig;
    rho_live[i] = rho;
    rec.rho(i) = (T)rho;
    if (P.diag) ((T*)B.sigma)[i] = sig;
  }
}

template <int D, class T>
__global__ void __launch_bounds__(256, kMinBlocks<T>) k_density_summation(Params P, DevBuffers B,
                                                                          KC<T> k, int gated) {
  DevScalars* sc = B.sc;
  if (gated && !sc->new_adv) return;
  density_summation_range<D, T>(P, B, k, sc, blockIdx.x * blockDim.x + threadIdx.x, P.n,
                                gridDim.x * blockDim.x);
}

// Density summation of the mixed path: exact integer pair distances from the
// fixed-point offsets of the rebuild and the kernel in double-float, so the
// density (and through c0^2 the pressure) keeps double-precision accuracy
// while every operation runs on the FP32 / integer pipes.
template <int D>
__device__ __forceinline__ unsigned long long fx_r2(const typename FxRec<D>::V& a,
                                                    const typename FxRec<D>::V& b, int dx, int dy,
                                                    int dz) {
  const long long ex = (a.x - dx * (int)kFxOne) - b.x;
  const long long ey = (a.y - dy * (int)kFxOne) - b.y;
  unsigned long long R2 = (unsigned long long)(ex * ex) + (unsigned long long)(ey * ey);
  if constexpr (D == 3) {
    const long long ez = (a.z - dz * (int)kFxOne) - b.z;
    R2 += (unsigned long long)(ez * ez);
  }
  return R2;
}

template <int D, class Slots>
__device__ __forceinline__ void density_summation_fx_slots(const Params& P, const DevBuffers& B,
                                                           DevScalars* sc, const Slots& slots) {
  using R = Rec<D, float>;
  using FV = typename FxRec<D>::V;
  const bool use_list = list_ok(P, sc, sc->drift_bad_p, sc->t_reb);
  double* rho_live = sc->par ? B.rho[1] : B.rho[0];
  const FV* __restrict__ rec = (const FV*)B.recI;
  const FV* __restrict__ wrec = (const FV*)B.wallI;
  const RecArr<D, float> lrec(B, 0);
  const uint32_t* __restrict__ keys = B.binned;
  const unsigned long long cut2 = 1ull << (2 * kFxShift);
  slots.each([&](const int i) {
    const Cell ci = decode(keys[i], P);
    const FV oi = rec[i];
    dfl sig = {1.0f, 0.0f};  // self first: shape(0) = 1, no term is larger
    visit_neighbours<D>(P, B, ci, i, use_list,
                        [&](int j, int dx, int dy, int dz, bool w, auto may_self) {
      if (may_self && !w && j == i) return;
      const unsigned long long R2 = fx_r2<D>(oi, w ? wrec[j] : rec[j], dx, dy, dz);
      if (R2 < cut2) sig = df_acc(sig, wendland_shape_fx(R2));
    });
    sig = fast_two_sum(sig.hi, sig.lo);
    const double sigma = P.walpha * ((double)sig.hi + (double)sig.lo);
    const double rho = reinit_density(P, sigma, rho_live[i]);
    if (P.variant & kVariantTransport) B.sigma64[i] = sigma;
    rho_live[i] = rho;
    lrec.rho(i) = (float)rho;
    if (P.diag) ((float*)B.sigma)[i] = (float)sigma;
  });
}

template <int D>
__device__ __forceinline__ void density_summation_fx_range(const Params& P, const DevBuffers& B,
                                                           DevScalars* sc, int i, int end,
                                                           int stride) {
  density_summation_fx_slots<D>(P, B, sc, StrideSlots{i, end, stride});
}

template <int D, bool kUnits = false>
__global__ void __launch_bounds__(256, 4) k_density_summation_fx(Params P, DevBuffers B,
                                                                 int gated) {
  DevScalars* sc = B.sc;
  if (gated && !sc->new_adv) return;
  if constexpr (kUnits)
    density_summation_fx_slots<D>(
        P, B, sc, UnitSlots{B.units, B.unit_ctr + 3 * B.parts, B.parts, (P.n + 31) >> 5, P.n});
  else
    density_summation_fx_range<D>(P, B, sc, blockIdx.x * blockDim.x + threadIdx.x, P.n,
                                  gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------
// Transport-velocity (particle-shifting) correction, once per advection step
// after the density summation (a method variant): every particle with full
// kernel support (sigma >= 0.95 sigma0, decided in double like the density)
// moves by -C h^2 sum_j V_j grad_i W_ij, C = 0.2, over fluid (V_j = m / rho_j)
// and wall (dp^dim) neighbours.  The walk only computes the shifts (into the
// prior-acceleration arrays, which the viscous stage overwrites next); the
// apply pass moves the particles and their records, so every shift uses the
// positions before any of them.
template <int D, class T>
__device__ __forceinline__ void transport_range(const Params& P, const DevBuffers& B,
                                                const KC<T>& k, DevScalars* sc, int i, int end,
                                                int stride,
                                     const ShiftTable* tab) {
  using R = Rec<D, T>;
  const bool use_list = list_ok(P, sc, sc->drift_bad_p, sc->t_reb);
  const RecArr<D, T> rec(B, 0);
  const uint32_t* __restrict__ keys = B.binned;
  T* d0 = (T*)B.aprior[0];
  T* d1 = (T*)B.aprior[1];
  T* d2 = (T*)B.aprior[2];
  const T wallV = (T)P.V;
  const T coef = (T)(-0.2 * P.h * P.h);
  for (; i < end; i += stride) {
    T gx = 0, gy = 0, gz = 0;
    if (B.sigma64[i] >= 0.95 * P.sigma0) {
      const Cell ci = decode(keys[i], P);
      const typename R::PV pi = rec.P(i);
      PairGeo<D, T> G{rec, (const typename WallRec<D, T>::WV*)B.wallP, R::px(pi), R::py(pi),
                      R::pz(pi), k.cs};
      visit_neighbours<D, Local<T>::kLocal>(
          P, B, ci, i, use_list, [&](int j, auto dx, auto dy, auto dz, bool w, auto may_self) {
        T rx, ry, rz;
        typename R::PV pj;
        typename R::SV sj;
        if (w) {
          G.rel_wall(G.wall[j], dx, dy, dz, rx, ry, rz);
        } else {
          rec.gather(j, pj, sj);
          G.rel_rec(pj, dx, dy, dz, rx, ry, rz);
        }
        const T r2 = r2_of(rx, ry, rz);
        if (!(r2 < k.r2max) || (may_self && !w && j == i)) return;
        const T r = sqrt(r2);
        T f;
        if (w) {
          f = wallV * wendland_dr(k, r) / r;
        } else {
          f = div_t(k.m, R::rho(pj, sj)) * wendland_dr(k, r) / r;
        }
        gx += f * rx;
        gy += f * ry;
        gz += f * rz;
      }, tab);
    }
    d0[i] = coef * gx;
    d1[i] = coef * gy;
    if (D == 3) d2[i] = coef * gz;
  }
}

template <int D, class T>
__global__ void __launch_bounds__(256, kMinBlocks<T>) k_transport(Params P, DevBuffers B, KC<T> k,
                                                                  int gated) {
  DevScalars* sc = B.sc;
  if (!(P.variant & kVariantTransport) || (gated && !sc->new_adv)) return;
  __shared__ ShiftTable tab;
  if constexpr (Local<T>::kLocal) fill_shift_table(tab);
  transport_range<D, T>(P, B, k, sc, blockIdx.x * blockDim.x + threadIdx.x, P.n,
                        gridDim.x * blockDim.x, &tab);
}

// Apply the shifts: positions (FP64 state) and the position records of
// buffer 0; a particle shifted out of its drift budget clears the lists for
// the viscous loop and the rest of the advection step.
template <int D, class T>
__device__ __forceinline__ void transport_apply_range(const Params& P, const DevBuffers& B,
                                                      DevScalars* sc, int i, int end,
                                                      int stride) {
  using R = Rec<D, T>;
  const Live<T> S = live<T>(B, sc->par);
  const RecArr<D, T> rec(B, 0);
  const uint32_t* __restrict__ keys = B.binned;
  const T* d0 = (const T*)B.aprior[0];
  const T* d1 = (const T*)B.aprior[1];
  const T* d2 = (const T*)B.aprior[2];
  int drift = 0;
  for (; i < end; i += stride) {
    const double sx = (double)d0[i], sy = (double)d1[i], sz = D == 3 ? (double)d2[i] : 0.0;
    const double x = S.x0[i] + sx, y = S.x1[i] + sy, z = D == 3 ? S.x2[i] + sz : 0.0;
    S.x0[i] = x;
    S.x1[i] = y;
    if (D == 3) S.x2[i] = z;
    T ox, oy, oz;
    Local<T>::enc(P, B.ctab, decode(keys[i], P), x, y, z, ox, oy, oz);
    drift |= drifted<D, T>(B, i, ox, oy, oz);
    typename R::PV p = rec.P(i);
    R::set_pos(p, ox, oy, oz);
    rec.P(i) = p;
  }
  // shifted positions, read by the viscous loop: outside a budget -> no lists
  flag_drift(&sc->drift_bad_p, drift);
}

template <int D, class T>
__global__ void k_transport_apply(Params P, DevBuffers B, int gated) {
  DevScalars* sc = B.sc;
  if (!(P.variant & kVariantTransport) || (gated && !sc->new_adv)) return;
  transport_apply_range<D, T>(P, B, sc, blockIdx.x * blockDim.x + threadIdx.x, P.n,
                              gridDim.x * blockDim.x);
}

// Viscous force: reads records P, S of buffer 0 (S carries the new rho);
// writes a_prior = g + viscous acceleration.  A wall particle enters with the
// mirrored velocity 2 v_w - v_i, so its pair term carries 2 (v_i - v_w) (the
// factor folded into its volume).  Positions are those of the rebuild, so the
// lists are always usable here (unless one overflowed).
template <int D, class T, class Slots>
__device__ __forceinline__ void viscous_slots(const Params& P, const DevBuffers& B, const KC<T>& k,
                                              DevScalars* sc, const Slots& slots,
                                              const ShiftTable* tab) {
  using R = Rec<D, T>;
  const bool use_list = list_ok(P, sc, sc->drift_bad_p, sc->t_reb);
  const RecArr<D, T> rec(B, 0);
  const uint32_t* __restrict__ keys = B.binned;
  T* ap0 = (T*)B.aprior[0];
  T* ap1 = (T*)B.aprior[1];
  T* ap2 = (T*)B.aprior[2];
  const T wallV2 = (T)(2.0 * P.V);
  const bool moving = (P.variant & kVariantMovingWall) != 0;
  slots.each([&](const int i) {
    const Cell ci = decode(keys[i], P);
    typename R::PV pi;
    typename R::SV si;
    rec.gather(i, pi, si);
    PairGeo<D, T> G{rec, (const typename WallRec<D, T>::WV*)B.wallP, R::px(pi), R::py(pi),
                    R::pz(pi), k.cs};
    const T vxi = R::vx(pi, si), vyi = R::vy(pi, si), vzi = R::vz(pi, si);
    T ax = 0, ay = 0, az = 0;
    visit_neighbours<D, Local<T>::kLocal && !kShiftBits<D>,
                     Local<T>::kLocal && kShiftBits<D>>(
        P, B, ci, i, use_list, [&](int j, auto dx, auto dy, auto dz, bool w, auto may_self) {
      T rx, ry, rz;
      typename R::PV pj;
      typename R::SV sj;
      if (w) {
        G.rel_wall(G.wall[j], dx, dy, dz, rx, ry, rz);
      } else {
        rec.gather(j, pj, sj);
        G.rel_rec(pj, dx, dy, dz, rx, ry, rz);
      }
      const T r2 = r2_of(rx, ry, rz);
      if (!(r2 < k.r2max) || (may_self && !w && j == i)) return;
      const T r = r2 * inv_sqrt_t(r2);
      const T t = T(1) + r * k.neg_inv_2h;
      // W'(r) / (r + eps) = (cdW/h) t^3 r / (r + eps); cdW/h applied per particle
      const T g = (t * t * t) * div_t(r, r + k.eps);
      if (w) {
        const T coef = wallV2 * g;
        T ux = vxi, uy = vyi, uz = vzi;
        if (moving) {
          using WR = WallRec<D, T>;
          const typename WR::WV vw = ((const typename WR::WV*)B.wall_vel)[j];
          ux -= vw.x;
          uy -= vw.y;
          uz -= WR::z(vw);
        }
        ax += coef * ux;
        ay += coef * uy;
        az += coef * uz;
      } else {
        const T coef = div_t(k.m, R::rho(pj, sj)) * g;
        ax += coef * (vxi - R::vx(pj, sj));
        ay += coef * (vyi - R::vy(pj, sj));
        az += coef * (vzi - R::vz(pj, sj));
      }
    }, tab);
    const T f = div_t(k.two_mu * (k.cdW * k.inv_h), R::rho(pi, si));
    ap0[i] = k.g[0] + f * ax;
    ap1[i] = k.g[1] + f * ay;
    if (D == 3) ap2[i] = k.g[2] + f * az;
  });
}

template <int D, class T>
__device__ __forceinline__ void viscous_range(const Params& P, const DevBuffers& B, const KC<T>& k,
                                              DevScalars* sc, int i, int end, int stride,
                                              const ShiftTable* tab) {
  viscous_slots<D, T>(P, B, k, sc, StrideSlots{i, end, stride}, tab);
}

template <int D, class T, bool kUnits = false>
__global__ void __launch_bounds__(256, kMinBlocks<T>) k_viscous(Params P, DevBuffers B, KC<T> k,
                                                                int gated) {
  DevScalars* sc = B.sc;
  if (gated && !sc->new_adv) return;
  __shared__ ShiftTable tab;
  if constexpr (Local<T>::kLocal && !kShiftBits<D>) fill_shift_table(tab);
  if constexpr (kUnits)
    viscous_slots<D, T>(
        P, B, k, sc, UnitSlots{B.units, B.unit_ctr + 4 * B.parts, B.parts, (P.n + 31) >> 5, P.n},
        &tab);
  else
    viscous_range<D, T>(P, B, k, sc, blockIdx.x * blockDim.x + threadIdx.x, P.n,
                        gridDim.x * blockDim.x, &tab);
}

// First half of the acoustic step; writes records of buffer 0.
template <int D, class T>
__device__ __forceinline__ void half1_range(const Params& P, const DevBuffers& B,
                                            DevScalars* sc, int i, int end, int stride) {
  using R = Rec<D, T>;
  const int par = sc->par;
  const double dt = sc->dt_ac;
  const double hdt = 0.5 * dt;
  const uint32_t* __restrict__ keys = B.binned;
  const RecArr<D, T> rec(B, 0);
  const Live<T> S = live<T>(B, par);
  int drift = 0;
  for (; i < end; i += stride) {
    double rho = S.rho[i] + hdt * (double)S.drho[i];
    double p = P.c0sq * (rho - P.rho0);
    double vx = S.v0[i], vy = S.v1[i], vz = D == 3 ? S.v2[i] : 0.0;
    double x = S.x0[i] + hdt * vx;
    double y = S.x1[i] + hdt * vy;
    double z = D == 3 ? S.x2[i] + hdt * vz : 0.0;
    S.rho[i] = rho;
    S.x0[i] = x;
    S.x1[i] = y;
    if (D == 3) S.x2[i] = z;
    T ox, oy, oz;
    Local<T>::enc(P, B.ctab, decode(keys[i], P), x, y, z, ox, oy, oz);
    rec.store(i, R::makeP(ox, oy, oz, (T)vx, (T)vy, (T)vz, (T)p),
              R::makeS((T)vx, (T)vy, (T)vz, (T)rho, (T)p));
    drift |= drifted<D, T>(B, i, ox, oy, oz);
  }
  // positions the pressure loop reads: outside a budget -> no lists for it
  flag_drift(&sc->drift_bad_p, drift);
}

template <int D, class T>
__global__ void k_half1(Params P, DevBuffers B) {
  // claim counters of this step's relaxation loops (brick order)
  if (B.units && blockIdx.x == 0)
    for (int t = threadIdx.x; t < 2 * B.parts; t += blockDim.x) B.unit_ctr[t] = 0;
  half1_range<D, T>(P, B, B.sc, blockIdx.x * blockDim.x + threadIdx.x, P.n,
                    gridDim.x * blockDim.x);
}

// Whether the pressure and density-relaxation loops are compiled with the
// wall-velocity term: always for sliding walls; for walls at rest only in 3D.
// Both forms give the same results; measured on the 5.1 M 3D dam break and
// the 256 2D tanks, the 3D loops ran 0.8 % faster with the (untaken) term
// compiled in and the 2D loops, at their 48-register cap, 4 % slower.
template <int D>
inline bool wall_vel_code(int variant) {
  return (variant & kVariantMovingWall) != 0 || D == 3;
}

// Riemann pressure relaxation + kick + the drift that opens the density stage.
// Reads records of buffer 0, writes records of buffer 1.  kWallVel compiles
// in the (run-time checked) wall-velocity term of sliding walls
// (kVariantMovingWall); see wall_vel_code() for when it is left out.
template <int D, class T, bool kWallVel = true, bool kAccel = false, class Slots>
__device__ __forceinline__ void pressure_slots(const Params& P, const DevBuffers& B, const KC<T>& k,
                                               DevScalars* sc, const Slots& slots,
                                               const ShiftTable* tab) {
  using R = Rec<D, T>;
  const int par = sc->par;
  const double dt = sc->dt_ac;
  const double hdt = 0.5 * dt;
  const bool use_list =
      list_ok(P, sc, sc->drift_bad_p, sc->t0 + hdt);
  const RecArr<D, T> rec(B, 0), out(B, 1);
  const uint32_t* __restrict__ keys = B.binned;
  const T* ap0 = (const T*)B.aprior[0];
  const T* ap1 = (const T*)B.aprior[1];
  const T* ap2 = (const T*)B.aprior[2];
  const Live<T> S = live<T>(B, par);
  double vmax2 = 0.0;
  int bad = 0, drift = 0;
  slots.each([&](const int i) {
    const Cell ci = decode(keys[i], P);
    typename R::PV pi;
    typename R::SV si;
    rec.gather(i, pi, si);
    PairGeo<D, T> G{rec, (const typename WallRec<D, T>::WV*)B.wallP, R::px(pi), R::py(pi),
                    R::pz(pi), k.cs};
    const T vxi = R::vx(pi, si), vyi = R::vy(pi, si), vzi = R::vz(pi, si);
    const T p_i = R::pres(pi, si), rho_i = R::rho(pi, si);
    T ax = 0, ay = 0, az = 0;
    visit_neighbours<D, Local<T>::kLocal && !kShiftBits<D>, Local<T>::kLocal && kShiftBits<D>>(
        P, B, ci, i, use_list, [&](int j, auto dx, auto dy, auto dz, bool w, auto may_self) {
      T rx, ry, rz;
      typename R::PV pj;
      typename R::SV sj;
      if (w) {
        G.rel_wall(G.wall[j], dx, dy, dz, rx, ry, rz);
      } else {
        rec.gather(j, pj, sj);
        G.rel_rec(pj, dx, dy, dz, rx, ry, rz);
      }
      const T r2 = r2_of(rx, ry, rz);
      if (!(r2 < k.r2max) || (may_self && !w && j == i)) return;
      const T inv_r = inv_sqrt_t(r2);
      // dvr = (v_i - v_R) . r_ij, so U_L - U_R = -dvr / r
      T dvr, p_j, rho_j;
      if (w) {
        // mirrored state: p_w = p_i + rho_i (x_w - x_i).(g - a_w), x_w - x_i = -r_vec;
        // v_R = 2 v_w - v_i, so v_i - v_R = 2 (v_i - v_w)
        T gdot = -(rx * k.g[0] + ry * k.g[1] + rz * k.g[2]);
        if constexpr (kAccel) gdot += wall_acc_dot<D, T>(B, j, rx, ry, rz);
        p_j = p_i + rho_i * gdot;
        rho_j = k.rho0 + p_j * k.inv_c0sq;
        T d = vxi * rx + vyi * ry + vzi * rz;
        if constexpr (kWallVel)
          if (P.variant & kVariantMovingWall) d -= wall_vel_dot<D, T>(B, j, rx, ry, rz);
        dvr = T(2) * d;
      } else {
        dvr = (vxi - R::vx(pj, sj)) * rx + (vyi - R::vy(pj, sj)) * ry +
              (vzi - R::vz(pj, sj)) * rz;
        p_j = R::pres(pj, sj);
        rho_j = R::rho(pj, sj);
      }
      // [Z17] P* = (p_i + p_j)/2 + beta rbar c0 (U_L - U_R)/2 with
      // beta = min(3 max(U_L - U_R, 0) / c0, 1) and rbar = (rho_i + rho_j)/2:
      // for J = max(U_L - U_R, 0),  2 P* = p_i + p_j + (rho_i + rho_j) J min(3J/2, c0/2)
      const T J0 = -dvr * inv_r;
      const T J = J0 > T(0) ? J0 : T(0);
      T lim = T(1.5) * J;
      lim = lim < k.c0_half ? lim : k.c0_half;
      const T Ps2 = (p_i + p_j) + (rho_i + rho_j) * (J * lim);
      const T t = T(1) + (r2 * inv_r) * k.neg_inv_2h;
      const T f = Ps2 * div_t(T(1), rho_j) * (t * t * t);
      ax += f * rx;
      ay += f * ry;
      az += f * rz;
    }, tab);
    // -(2/rho_i) sum P* (m/rho_j) W' e_ij = (kP / rho_i) sum 2P* t^3 r_ij / rho_j
    const T s = div_t(k.kP, rho_i);
    ax *= s;
    ay *= s;
    az *= s;
    if (P.diag) {
      ((T*)B.acc[0])[i] = ax;
      ((T*)B.acc[1])[i] = ay;
      if (D == 3) ((T*)B.acc[2])[i] = az;
    }
    double vx = S.v0[i] + dt * (double)(ax + ap0[i]);
    double vy = S.v1[i] + dt * (double)(ay + ap1[i]);
    double vz = D == 3 ? S.v2[i] + dt * (double)(az + ap2[i]) : 0.0;
    double x = S.x0[i] + hdt * vx;
    double y = S.x1[i] + hdt * vy;
    double z = D == 3 ? S.x2[i] + hdt * vz : 0.0;
    S.v0[i] = vx;
    S.v1[i] = vy;
    S.x0[i] = x;
    S.x1[i] = y;
    if (D == 3) {
      S.v2[i] = vz;
      S.x2[i] = z;
    }
    double s2 = __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz));
    if (!(s2 <= 1e300)) bad = 1;  // NaN or overflow
    vmax2 = s2 > vmax2 ? s2 : vmax2;
    T ox, oy, oz;
    Local<T>::enc(P, B.ctab, ci, x, y, z, ox, oy, oz);
    out.store(i, R::makeP(ox, oy, oz, (T)vx, (T)vy, (T)vz, p_i),
              R::makeS((T)vx, (T)vy, (T)vz, rho_i, p_i));
    drift |= drifted<D, T>(B, i, ox, oy, oz);
  });
  vmax2 = warp_max(vmax2);
  __shared__ double wm[32];
  __syncthreads();  // the previous body call of this block has read wm
  if (threadIdx.x % 32 == 0) wm[threadIdx.x / 32] = vmax2;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&sc->flags, kFlagNonFinite);
  // positions the density relaxation reads: outside a budget -> no lists for it
  flag_drift(&sc->drift_bad_r, drift);
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x / 32); ++q) vmax2 = fmax(vmax2, wm[q]);
    if (!(vmax2 <= 1e300)) vmax2 = 1e300;
    atomicMax(&sc->vmax2_next, (unsigned long long)__double_as_longlong(vmax2));
  }
}

template <int D, class T, bool kWallVel = true, bool kAccel = false>
__device__ __forceinline__ void pressure_range(const Params& P, const DevBuffers& B, const KC<T>& k,
                                               DevScalars* sc, int i, int end, int stride,
                                               const ShiftTable* tab) {
  pressure_slots<D, T, kWallVel, kAccel>(P, B, k, sc, StrideSlots{i, end, stride}, tab);
}

// kUnits: the slots in brick order (one tank, 3D mixed), else strided.
template <int D, class T, bool kWallVel, bool kAccel = false, bool kUnits = false>
__global__ void __launch_bounds__(256, kMinBlocksPres<D, T>) k_pressure(Params P, DevBuffers B,
                                                                         KC<T> k) {
  __shared__ ShiftTable tab;
  if constexpr (Local<T>::kLocal && !kShiftBits<D>) fill_shift_table(tab);
  if constexpr (kUnits)
    pressure_slots<D, T, kWallVel, kAccel>(
        P, B, k, B.sc, UnitSlots{B.units, B.unit_ctr, B.parts, (P.n + 31) >> 5, P.n}, &tab);
  else
    pressure_range<D, T, kWallVel, kAccel>(P, B, k, B.sc, blockIdx.x * blockDim.x + threadIdx.x,
                                           P.n, gridDim.x * blockDim.x, &tab);
}

// Riemann density relaxation: reads records of buffer 1; drho and rho (state).
// kWallVel as for the pressure relaxation.
template <int D, class T, bool kWallVel = true, bool kAccel = false, class Slots>
__device__ __forceinline__ void density_relax_slots(const Params& P, const DevBuffers& B,
                                                    const KC<T>& k, DevScalars* sc,
                                                    const Slots& slots, const ShiftTable* tab) {
  using R = Rec<D, T>;
  const int par = sc->par;
  const double hdt = 0.5 * sc->dt_ac;
  const bool use_list =
      list_ok(P, sc, sc->drift_bad_r, sc->t0 + 2.0 * hdt);
  const RecArr<D, T> rec(B, 1);
  const uint32_t* __restrict__ keys = B.binned;
  const Live<T> S = live<T>(B, par);
  int bad = 0;
  slots.each([&](const int i) {
    const Cell ci = decode(keys[i], P);
    typename R::PV pi;
    typename R::SV si;
    rec.gather(i, pi, si);
    PairGeo<D, T> G{rec, (const typename WallRec<D, T>::WV*)B.wallP, R::px(pi), R::py(pi),
                    R::pz(pi), k.cs};
    const T vxi = R::vx(pi, si), vyi = R::vy(pi, si), vzi = R::vz(pi, si);
    const T p_i = R::pres(pi, si), rho_i = R::rho(pi, si);
    T sum = 0;
    visit_neighbours<D, Local<T>::kLocal && !kShiftBits<D>,
                     Local<T>::kLocal && kShiftBits<D>>(
        P, B, ci, i, use_list, [&](int j, auto dx, auto dy, auto dz, bool w, auto may_self) {
      T rx, ry, rz;
      typename R::PV pj;
      typename R::SV sj;
      if (w) {
        G.rel_wall(G.wall[j], dx, dy, dz, rx, ry, rz);
      } else {
        rec.gather(j, pj, sj);
        G.rel_rec(pj, dx, dy, dz, rx, ry, rz);
      }
      const T r2 = r2_of(rx, ry, rz);
      if (!(r2 < k.r2max) || (may_self && !w && j == i)) return;
      const T r = r2 * inv_sqrt_t(r2);
      const T t = T(1) + r * k.neg_inv_2h;
      // [Z17] U* = (U_L + U_R)/2 + riemann (p_i - p_j) / (2 rbar c0), so with
      // W'(r) e_ij = (cdW/h) t^3 r_ij the pair term -2 rho_i V_j W' (U_L - U*)
      // is kD rho_i t^3 B_ij / rho_j with
      //   B_ij = (v_i - v_j).r_ij + kappa2 r (p_i - p_j) / (rho_i + rho_j),
      // summed as t^3 (dvr S + kappa2 r (p_i - p_j)) / (rho_j S), S = rho_i + rho_j
      // (one reciprocal); at a wall v_j is the mirrored v_R = 2 v_w - v_i, whose
      // half-difference (v_i - v_R)/2 = v_i - v_w enters in full.
      T Bij, rho_j;
      if (w) {
        T gdot = -(rx * k.g[0] + ry * k.g[1] + rz * k.g[2]);
        if constexpr (kAccel) gdot += wall_acc_dot<D, T>(B, j, rx, ry, rz);
        const T pw_ = p_i + rho_i * gdot;
        rho_j = k.rho0 + pw_ * k.inv_c0sq;
        T d = vxi * rx + vyi * ry + vzi * rz;
        if constexpr (kWallVel)
          if (P.variant & kVariantMovingWall) d -= wall_vel_dot<D, T>(B, j, rx, ry, rz);
        const T sr = rho_i + rho_j;
        Bij = fma_t(T(2) * d, sr, (k.kappa2 * r) * (p_i - pw_)) * div_t(T(1), rho_j * sr);
      } else {
        rho_j = R::rho(pj, sj);
        const T dvr = (vxi - R::vx(pj, sj)) * rx + (vyi - R::vy(pj, sj)) * ry +
                      (vzi - R::vz(pj, sj)) * rz;
        const T sr = rho_i + rho_j;
        Bij = fma_t(dvr, sr, (k.kappa2 * r) * (p_i - R::pres(pj, sj))) * div_t(T(1), rho_j * sr);
      }
      sum = fma_t(t * t * t, Bij, sum);  // Bij here carries the 1 / rho_j
    }, tab);
    const T dr = k.kD * rho_i * sum;
    S.drho[i] = dr;
    double rho = S.rho[i] + hdt * (double)dr;
    if (!(fabs(rho) <= 1e300)) bad = 1;
    S.rho[i] = rho;
  });
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&sc->flags, kFlagNonFinite);
}

template <int D, class T, bool kWallVel = true, bool kAccel = false>
__device__ __forceinline__ void density_relax_range(const Params& P, const DevBuffers& B,
                                                    const KC<T>& k, DevScalars* sc, int i,
                                                    int end, int stride,
                                                    const ShiftTable* tab) {
  density_relax_slots<D, T, kWallVel, kAccel>(P, B, k, sc, StrideSlots{i, end, stride}, tab);
}

// One tank: block 0 also publishes this step's velocity maximum for the next
// step's schedule (a batch does that in its schedule kernel).
template <int D, class T, bool kWallVel, bool kAccel = false, bool kUnits = false>
__global__ void __launch_bounds__(256, kMinBlocksP<D, T>) k_density_relax(Params P, DevBuffers B,
                                                                          KC<T> k) {
  DevScalars* sc = B.sc;
  __shared__ ShiftTable tab;
  if constexpr (Local<T>::kLocal && !kShiftBits<D>) fill_shift_table(tab);
  if (blockIdx.x == 0 && threadIdx.x == 0) sc->vmax2_cur = sc->vmax2_next;
  if constexpr (kUnits)
    density_relax_slots<D, T, kWallVel, kAccel>(
        P, B, k, sc,
        UnitSlots{B.units, B.unit_ctr + B.parts, B.parts, (P.n + 31) >> 5, P.n}, &tab);
  else
    density_relax_range<D, T, kWallVel, kAccel>(P, B, k, sc, blockIdx.x * blockDim.x + threadIdx.x,
                                                P.n, gridDim.x * blockDim.x, &tab);
}

// Wall setup: gather sorted wall positions (double SoA for the parity kernel,
// records for the loops), ids and, for moving walls, the prescribed
// velocities from the unsorted staging copy.  Slot k of the sorted walls takes
// staging entry j, binned in cell `key` of its tank's grid; (wx, wy, wz) is
// the double SoA of all sorted walls; uv the velocity SoA staging (x | y | z,
// vstride apart), read only when wall_vel is set.
template <int D, class T>
__device__ __forceinline__ void wall_slot(const Params& P, const DevBuffers& B,
                                          const double* __restrict__ ux,
                                          const double* __restrict__ uy,
                                          const double* __restrict__ uz, double* wx, double* wy,
                                          double* wz, const double* __restrict__ uv,
                                          size_t vstride, int k, uint32_t j, uint32_t key) {
  using WR = WallRec<D, T>;
  typename WR::WV* out = (typename WR::WV*)B.wallP;
  if (!SPH_DBG_IN(B, j, 0, vstride)) return;
  double x = ux[j], y = uy[j], z = D == 3 ? uz[j] : 0.0;
  wx[k] = x;
  wy[k] = y;
  if (D == 3) wz[k] = z;
  B.wall_id[k] = j;
  if (B.wall_key) B.wall_key[k] = key;
  T ox, oy, oz;
  const Cell ck = decode(key, P);
  Local<T>::enc(P, B.ctab, ck, x, y, z, ox, oy, oz);
  out[k] = WR::make(ox, oy, oz);
  if (B.wall_vel)
    ((typename WR::WV*)B.wall_vel)[k] =
        WR::make((T)uv[j], (T)uv[vstride + j], D == 3 ? (T)uv[2 * vstride + j] : T(0));
  if constexpr (Local<T>::kLocal)
    ((typename FxRec<D>::V*)B.wallI)[k] = fx_encode<D>(P, ck, x, y, z);
}

template <int D, class T>
__global__ void k_wall_gather(Params P, DevBuffers B, const double* __restrict__ ux,
                              const double* __restrict__ uy, const double* __restrict__ uz,
                              double* wx, double* wy, double* wz, const double* uv, int gated) {
  if (gated && !B.sc->new_adv) return;
  const uint32_t* perm = B.vals[B.sorted_buf];
  const uint32_t* keys = B.keys[B.sorted_buf];
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < P.nw; k += gridDim.x * blockDim.x)
    wall_slot<D, T>(P, B, ux, uy, uz, wx, wy, wz, uv, (size_t)P.nw, k, perm[k], keys[k]);
}

// Translating walls.  k_wall_place writes every wall's position at the
// binning time into wall_io: x0 + t v0 for a translating wall, x0 for the
// others.  The binning time is the step's start time at a rebuild
// (kBinAtStepStart), the current time (kBinNow), or the time of the last
// rebuild (kBinAtRebuild, when a saved state is restored).
constexpr int kBinAtStepStart = 0, kBinNow = 1, kBinAtRebuild = 2;

// Kinematics of translating wall u (user order) along axis c at time t:
// x0 + v t + A sin(omega t), v + A omega cos(omega t), -A omega^2 sin(omega t).
struct WallKin {
  double sn, cs, w;
  __device__ WallKin(const Params& P, double t)
      : sn(sin(P.wall_omega * t)), cs(cos(P.wall_omega * t)), w(P.wall_omega) {}
  __device__ double x(const DevBuffers& B, size_t nw, size_t u, int c, double t) const {
    double x = B.wall_x0[c * nw + u] + t * B.wall_v0[c * nw + u];
    if (B.wall_amp) x += B.wall_amp[c * nw + u] * sn;
    return x;
  }
  __device__ double v(const DevBuffers& B, size_t nw, size_t u, int c) const {
    double v = B.wall_v0[c * nw + u];
    if (B.wall_amp) v += B.wall_amp[c * nw + u] * w * cs;
    return v;
  }
  __device__ double a(const DevBuffers& B, size_t nw, size_t u, int c) const {
    return B.wall_amp ? -B.wall_amp[c * nw + u] * w * w * sn : 0.0;
  }
};

template <int D>
__global__ void k_wall_place(Params P, DevBuffers B, int gated, int when) {
  DevScalars* sc = B.sc;
  if (gated && !sc->new_adv) return;
  const double t = when == kBinNow ? sc->t : (when == kBinAtRebuild ? sc->t_reb : sc->t0);
  const WallKin K(P, t);
  const size_t nw = (size_t)P.nw;
  for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < nw;
       u += (size_t)gridDim.x * blockDim.x) {
    const bool moves = B.wall_moves && B.wall_moves[u] && B.wall_v0;
    for (int c = 0; c < 3; ++c)
      B.wall_io[c * nw + u] = moves ? K.x(B, nw, u, c, t) : B.wall_x0[c * nw + u];
  }
}

// Moves the translating walls (sorted slots) to a time: the fluid's after
// the first half-drift (kMoveHalf: t0 + dt/2) or the second (kMoveFull:
// t0 + dt), the step's start (kMoveStepStart, after a rebuild) or now
// (kMoveNow); their records stay relative to the cell they were binned in.
// Oscillating walls also get their velocity and acceleration at that time.
constexpr int kMoveHalf = 1, kMoveFull = 0, kMoveStepStart = 2, kMoveNow = 3;

template <int D, class T>
__global__ void k_wall_move(Params P, DevBuffers B, int when) {
  using WR = WallRec<D, T>;
  const DevScalars* sc = B.sc;
  const double t = when == kMoveHalf   ? sc->t0 + 0.5 * sc->dt_ac
                   : when == kMoveFull ? sc->t0 + sc->dt_ac
                   : when == kMoveNow  ? sc->t
                                       : sc->t0;
  const WallKin K(P, t);
  const size_t nw = (size_t)P.nw;
  typename WR::WV* out = (typename WR::WV*)B.wallP;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < nw;
       k += (size_t)gridDim.x * blockDim.x) {
    const uint32_t u = B.wall_id[k];
    if (!B.wall_moves || !B.wall_v0 || !B.wall_moves[u]) continue;
    const double x = K.x(B, nw, u, 0, t);
    const double y = K.x(B, nw, u, 1, t);
    const double z = D == 3 ? K.x(B, nw, u, 2, t) : 0.0;
    B.wall_xyz[k] = x;
    B.wall_xyz[nw + k] = y;
    if (D == 3) B.wall_xyz[2 * nw + k] = z;
    T ox, oy, oz;
    Local<T>::enc(P, B.ctab, decode(B.wall_key[k], P), x, y, z, ox, oy, oz);
    out[k] = WR::make(ox, oy, oz);
    if (B.wall_amp) {
      ((typename WR::WV*)B.wall_vel)[k] =
          WR::make((T)K.v(B, nw, u, 0), (T)K.v(B, nw, u, 1), D == 3 ? (T)K.v(B, nw, u, 2) : T(0));
      ((typename WR::WV*)B.wall_acc)[k] =
          WR::make((T)K.a(B, nw, u, 0), (T)K.a(B, nw, u, 1), D == 3 ? (T)K.a(B, nw, u, 2) : T(0));
    }
  }
}

// The same at the step's start, for the gated rebuild of the plain launch
// sequence: runs only when the step begins an advection step.
template <int D, class T>
__global__ void k_wall_move_gated(Params P, DevBuffers B) {
  if (!B.sc->new_adv) return;
  // one block-uniform decision, then the same body
  using WR = WallRec<D, T>;
  const DevScalars* sc = B.sc;
  const double t = sc->t0;
  const WallKin K(P, t);
  const size_t nw = (size_t)P.nw;
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < nw;
       k += (size_t)gridDim.x * blockDim.x) {
    const uint32_t u = B.wall_id[k];
    if (!B.wall_moves || !B.wall_v0 || !B.wall_amp || !B.wall_moves[u]) continue;
    ((typename WR::WV*)B.wall_vel)[k] =
        WR::make((T)K.v(B, nw, u, 0), (T)K.v(B, nw, u, 1), D == 3 ? (T)K.v(B, nw, u, 2) : T(0));
    ((typename WR::WV*)B.wall_acc)[k] =
        WR::make((T)K.a(B, nw, u, 0), (T)K.a(B, nw, u, 1), D == 3 ? (T)K.a(B, nw, u, 2) : T(0));
  }
}

// ---------------------------------------------------------------------------
inline int grid_for(int n, int block, int cap) {
  int b = (n + block - 1) / block;
  if (b > cap) b = cap;
  return b < 1 ? 1 : b;
}

// Records ev[k] before stage k (and ev[kStages] after the last) when given.
inline void mark(cudaEvent_t* ev, int k, cudaStream_t s) {
  if (ev) cudaEventRecord(ev[k], s);
}

// Translating walls binned again: placed at the binning time, keys, a stable
// sort in the wall buffers, the gather of records and ids, the wall offsets.
// kBinAtRebuild then moves the walls on to the current time, as the steps
// since that rebuild left them.
template <int D, class T>
void enqueue_wall_rebin_t(const StageArgs& a, cudaStream_t s, int gated, int when) {
  const Params& P = a.P;
  const LaunchCfg& L = a.L;
  if (P.nw <= 0) return;
  DevBuffers W = a.B;
  const size_t nw = (size_t)P.nw;
  const int gw = grid_for(P.nw, 256, L.blocks_stream);
  k_wall_place<D><<<gw, 256, 0, s>>>(P, W, gated, when);
  const double* xs[3] = {W.wall_io, W.wall_io + nw, W.wall_io + 2 * nw};
  launch_cell_keys(P, L, xs, W.wkeys[0], W.wvals[0], P.nw, W.sc, gated, W.digit_total, s);
  const int cur = launch_radix_sort(L, W.wkeys, W.wvals, P.nw, W.wtile_hist, W.digit_total, W.sc,
                                    gated, s);
  W.keys[0] = W.wkeys[0];
  W.keys[1] = W.wkeys[1];
  W.vals[0] = W.wvals[0];
  W.vals[1] = W.wvals[1];
  W.sorted_buf = cur;
  k_wall_gather<D, T><<<gw, 256, 0, s>>>(P, W, xs[0], xs[1], xs[2], W.wall_xyz,
                                         W.wall_xyz + nw, W.wall_xyz + 2 * nw, W.wall_v0, gated);
  launch_cell_offsets(W.wkeys[cur], P.nw, P.ncell, W.wall_cb, W.sc, gated, 0, s);
  if (when == kBinAtRebuild) {
    k_wall_move<D, T><<<gw, 256, 0, s>>>(P, W, kMoveFull);
  } else if (P.variant & kVariantAccelWall) {
    // velocities and accelerations of oscillating walls at the binning time
    // (the gather wrote the constant part); gated like the rebuild
    if (!gated || when != kBinAtStepStart)
      k_wall_move<D, T><<<gw, 256, 0, s>>>(P, W, when == kBinNow ? kMoveNow : kMoveStepStart);
    else
      k_wall_move_gated<D, T><<<gw, 256, 0, s>>>(P, W);
  }
}

// Grid of one resident wave of a loop kernel that takes its work from
// UnitSlots (blocks of L.block_loop threads on every multiprocessor).
template <class K>
int one_wave(K kernel, const LaunchCfg& L) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, L.block_loop, 0) != cudaSuccess ||
      nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  return nb * L.sms;
}

template <int D, class T>
void enqueue_units(const StageArgs& a, cudaStream_t s, int gated) {
  const Params& P = a.P;
  if (D != 3 || !Local<T>::kLocal || !a.B.units || P.n <= 0) return;
  const int ng = (P.n + 31) >> 5;
  const int gs = grid_for(ng, 256, a.L.blocks_stream);
  const int nclear = max((int)brick_count(P) + 1, 3 * a.B.parts);
  k_units_clear<D><<<grid_for(nclear, 256, a.L.blocks_stream), 256, 0, s>>>(P, a.B, gated);
  k_units_count<D><<<gs, 256, 0, s>>>(P, a.B, gated);
  k_units_scan<D><<<1, kUnitScanThreads, 0, s>>>(P, a.B, gated);
  k_units_scatter<D><<<gs, 256, 0, s>>>(P, a.B, gated);
}

template <int D, class T>
void enqueue_rebuild(const StageArgs& a, cudaStream_t s, int gated, cudaEvent_t* ev) {
  const Params& P = a.P;
  const LaunchCfg& L = a.L;
  DevBuffers B = a.B;
  uint32_t* keys[2] = {B.keys[0], B.keys[1]};
  uint32_t* vals[2] = {B.vals[0], B.vals[1]};
  mark(ev, kStageKeys, s);
  launch_cell_keys_par(P, L, B.x, keys[0], vals[0], P.n, B.sc, gated, B.digit_total, s);
  mark(ev, kStageSort, s);
  B.sorted_buf = launch_radix_sort(L, keys, vals, P.n, B.tile_hist, B.digit_total, B.sc, gated, s);
  mark(ev, kStageReorder, s);
  k_reorder<D, T><<<grid_for(P.n, L.block_stream, L.blocks_stream), L.block_stream, 0, s>>>(
      P, B, gated);
  mark(ev, kStageOffsets, s);
  launch_cell_offsets(B.keys[B.sorted_buf], P.n, P.ncell, B.cell_begin, B.sc, gated, 1, s);
  enqueue_units<D, T>(a, s, gated);
  if (P.variant & kVariantTranslatingWall) enqueue_wall_rebin_t<D, T>(a, s, gated, kBinAtStepStart);
}

// Stages after the rebuild of an advection step; gated: each kernel returns at
// once unless the step begins an advection step.
template <int D, class T>
void enqueue_advection_loops(const StageArgs& a, cudaStream_t s, int gated, cudaEvent_t* ev) {
  const Params& P = a.P;
  const LaunchCfg& L = a.L;
  const DevBuffers& B = a.B;
  const KC<T> k = make_kc<T>(P);
  const int gl = grid_for(P.n, L.block_loop, L.blocks_loop);
  constexpr bool kU = D == 3 && Local<T>::kLocal;  // brick order when B.units is set
  const bool units = kU && B.units;
  mark(ev, kStageDensitySum, s);
  if (units)
    k_build_lists<D, T, kU><<<one_wave(k_build_lists<D, T, kU>, L), L.block_loop, 0, s>>>(P, B, k,
                                                                                       gated);
  else
    k_build_lists<D, T><<<gl, L.block_loop, 0, s>>>(P, B, k, gated);
  if constexpr (Local<T>::kLocal) {
    if (units)
      k_density_summation_fx<D, kU><<<one_wave(k_density_summation_fx<D, kU>, L), L.block_loop, 0,
                                      s>>>(P, B, gated);
    else
      k_density_summation_fx<D><<<gl, L.block_loop, 0, s>>>(P, B, gated);
  } else {
    k_density_summation<D, T><<<gl, L.block_loop, 0, s>>>(P, B, k, gated);
  }
  if (P.variant & kVariantTransport) {
    k_transport<D, T><<<gl, L.block_loop, 0, s>>>(P, B, k, gated);
    k_transport_apply<D, T><<<grid_for(P.n, L.block_stream, L.blocks_stream), L.block_stream, 0,
                              s>>>(P, B, gated);
  }
  mark(ev, kStageViscous, s);
  if (units)
    k_viscous<D, T, kU><<<one_wave(k_viscous<D, T, kU>, L), L.block_loop, 0, s>>>(P, B, k, gated);
  else
    k_viscous<D, T><<<gl, L.block_loop, 0, s>>>(P, B, k, gated);
}

template <int D, class T>
void enqueue_acoustic_t(const StageArgs& a, cudaStream_t s, cudaEvent_t* ev = nullptr) {
  const Params& P = a.P;
  const LaunchCfg& L = a.L;
  const DevBuffers& B = a.B;
  const KC<T> k = make_kc<T>(P);
  const int gl = grid_for(P.n, L.block_loop, L.blocks_loop);
  const int gs = grid_for(P.n, L.block_stream, L.blocks_stream);
  const bool translating = (P.variant & kVariantTranslatingWall) && P.nw > 0;
  const int gw = grid_for(P.nw, 256, L.blocks_stream);
  mark(ev, kStageHalf1, s);
  k_half1<D, T><<<gs, L.block_stream, 0, s>>>(P, B);
  if (translating) k_wall_move<D, T><<<gw, 256, 0, s>>>(P, B, kMoveHalf);
  mark(ev, kStagePressure, s);
  const bool wall_vel = wall_vel_code<D>(P.variant);
  const bool accel = (P.variant & kVariantAccelWall) != 0;
  constexpr bool kU = D == 3 && Local<T>::kLocal;  // brick order when B.units is set
  const bool units = kU && B.units;
  if (accel)
    k_pressure<D, T, true, true><<<gl, L.block_loop, 0, s>>>(P, B, k);
  else if (wall_vel && units)
    k_pressure<D, T, true, false, kU><<<one_wave(k_pressure<D, T, true, false, kU>, L),
                                        L.block_loop, 0, s>>>(P, B, k);
  else if (wall_vel)
    k_pressure<D, T, true><<<gl, L.block_loop, 0, s>>>(P, B, k);
  else if (units)
    k_pressure<D, T, false, false, kU><<<one_wave(k_pressure<D, T, false, false, kU>, L),
                                         L.block_loop, 0, s>>>(P, B, k);
  else
    k_pressure<D, T, false><<<gl, L.block_loop, 0, s>>>(P, B, k);
  if (translating) k_wall_move<D, T><<<gw, 256, 0, s>>>(P, B, kMoveFull);
  mark(ev, kStageDensityRelax, s);
  if (accel)
    k_density_relax<D, T, true, true><<<gl, L.block_loop, 0, s>>>(P, B, k);
  else if (wall_vel && units)
    k_density_relax<D, T, true, false, kU><<<one_wave(k_density_relax<D, T, true, false, kU>, L),
                                             L.block_loop, 0, s>>>(P, B, k);
  else if (wall_vel)
    k_density_relax<D, T, true><<<gl, L.block_loop, 0, s>>>(P, B, k);
  else if (units)
    k_density_relax<D, T, false, false, kU><<<one_wave(k_density_relax<D, T, false, false, kU>, L),
                                              L.block_loop, 0, s>>>(P, B, k);
  else
    k_density_relax<D, T, false><<<gl, L.block_loop, 0, s>>>(P, B, k);
  mark(ev, kStages, s);
}

// One acoustic step as a plain launch sequence (the rebuild stages gated).
template <int D, class T>
void enqueue_step_t(const StageArgs& a, cudaStream_t s, cudaEvent_t* ev) {
  mark(ev, kStageControl, s);
  launch_control(a.P, a.B.sc, s);
  enqueue_rebuild<D, T>(a, s, 1, ev);
  enqueue_advection_loops<D, T>(a, s, 1, ev);
  enqueue_acoustic_t<D, T>(a, s, ev);
}

// The body of the graph's conditional node: the same stages, ungated.
template <int D, class T>
void enqueue_advection_t(const StageArgs& a, cudaStream_t s) {
  enqueue_rebuild<D, T>(a, s, 0, nullptr);
  enqueue_advection_loops<D, T>(a, s, 0, nullptr);
}

// Lists for a restored state: built from the positions as they stand, with
// budgets b_k + d_k, d_k the drift since the rebuild so far.  A pair left out
// is farther than 2h + b_i + d_i + b_j + d_j now; a particle moves at most
// d_k + b_k from here before it leaves its budget, so the pair stays farther
// than 2h while the stored budgets hold -- the condition the loops check.
// A list's sums depend only on the pairs within 2h, visited in candidate
// order: the same sums as the lists of the rebuild.
template <int D, class T>
__global__ void k_restore_budgets(Params P, DevBuffers B) {
  const Live<T> S = live<T>(B, B.sc->par);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
    T ox, oy, oz;
    Local<T>::enc(P, B.ctab, decode(B.binned[i], P), S.x0[i], S.x1[i],
                  D == 3 ? S.x2[i] : 0.0, ox, oy, oz);
    const double dx = (double)ox - (double)((const T*)B.xreb[0])[i];
    const double dy = (double)oy - (double)((const T*)B.xreb[1])[i];
    const double dz = D == 3 ? (double)oz - (double)((const T*)B.xreb[2])[i] : 0.0;
    // b + d with a margin for the record frame's rounding, rounded up
    const float grown =
        __double2float_ru(1.001 * ((double)B.bud[i] + sqrt(dx * dx + dy * dy + dz * dz)));
    ((typename Vec4<T>::type*)B.brec)[i] = build_rec<D, T>(ox, oy, oz, (T)grown);
  }
}

template <int D, class T>
void enqueue_restore_lists_t(const StageArgs& a, cudaStream_t s) {
  const Params& P = a.P;
  const LaunchCfg& L = a.L;
  if (!P.use_list || P.n <= 0) return;
  const int gs = grid_for(P.n, L.block_stream, L.blocks_stream);
  k_encode_records<D, T><<<gs, L.block_stream, 0, s>>>(P, a.B);
  // build records: current positions, budgets b + (drift so far)
  k_restore_budgets<D, T><<<gs, L.block_stream, 0, s>>>(P, a.B);
  k_build_lists<D, T><<<grid_for(P.n, L.block_loop, L.blocks_loop), L.block_loop, 0, s>>>(
      P, a.B, make_kc<T>(P), 0);
}

template <int D, class T>
void enqueue_initial_sort_t(const StageArgs& a, cudaStream_t s) {
  enqueue_rebuild<D, T>(a, s, 0, nullptr);
}

template <int D, class T>
void enqueue_wall_setup_t(const StageArgs& a, cudaStream_t s) {
  const Params& P = a.P;
  const LaunchCfg& L = a.L;
  DevBuffers B = a.B;
  const double* ux = B.io;
  const double* uy = B.io + P.nw;
  const double* uz = B.io + 2 * (size_t)P.nw;
  double* wx = B.wall_xyz;
  double* wy = wx + P.nw;
  double* wz = wy + P.nw;
  const double* xs[3] = {ux, uy, uz};
  uint32_t* keys[2] = {B.keys[0], B.keys[1]};
  uint32_t* vals[2] = {B.vals[0], B.vals[1]};
  launch_cell_keys(P, L, xs, keys[0], vals[0], P.nw, nullptr, 0, B.digit_total, s);
  B.sorted_buf = launch_radix_sort(L, keys, vals, P.nw, B.tile_hist, B.digit_total, B.sc, 0, s);
  // velocity staging after the positions: io + 3 nw (x | y | z)
  const double* uv = B.wall_vel ? B.io + 3 * (size_t)P.nw : nullptr;
  k_wall_gather<D, T><<<grid_for(P.nw, 256, L.blocks_stream), 256, 0, s>>>(P, B, ux, uy, uz, wx,
                                                                          wy, wz, uv, 0);
  launch_cell_offsets(B.keys[B.sorted_buf], P.nw, P.ncell, B.wall_cb, B.sc, 0, 0, s);
}

}  // namespace stages
}  // namespace sphgb
