// Standalone neighbour search (sph_nsearch_*): the cell-linked-list build of
// the paper (cell keys, device radix sort, reorder, cell offsets; section
// "Cell linked-list, direct search and sorting") followed by one direct-search
// density pass, over caller-provided device positions in float or double.
// The density pass takes the sorted slots in brick order (the 32-slot groups
// sorted by brick of 4 x 4 x 4 cells, one run per multiprocessor), as the
// simulation's loops do.
// Each stage is timed with CUDA events on the object's stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

#include "sph.h"
#include "sph_internal.cuh"
#include "sph_stages.cuh"

using namespace sphgb;

struct sph_nsearch {
  Params P{};
  LaunchCfg L{};
  int fp32 = 0;  // positions are float
  sph_allocator alloc{};
  bool has_alloc = false;
  cudaStream_t user_stream = nullptr, stream = nullptr;
  cudaEvent_t ev[6] = {};
  size_t cap = 0;
  struct Blk {
    void* p;
    size_t b;
  };
  std::vector<Blk> blocks, fixed;
  uint32_t *keys[2] = {}, *vals[2] = {}, *tile_hist = nullptr, *digit_total = nullptr,
           *cell_begin = nullptr;
  void* sp = nullptr;  // sorted positions, packed (x, y, z, 0) of the position type
  void* pk = nullptr;  // the same packing in input order (written with the keys)
  double* sigma = nullptr;
  // brick processing order of the density pass (the one-tank loops' scheme):
  // DevBuffers fields units, unit_brick, brick_start, brick_fill, unit_ctr, parts
  DevBuffers U{};
  int sorted = 0;
  size_t n = 0;
};

namespace {

constexpr double kPiN = 3.14159265358979323846;

void* ns_alloc(sph_nsearch* s, size_t bytes, std::vector<sph_nsearch::Blk>& list) {
  bytes = (bytes + 255) & ~(size_t)255;
  if (!bytes) bytes = 256;
  void* p = nullptr;
  if (s->has_alloc) {
    p = s->alloc.alloc(bytes, (void*)s->stream, s->alloc.user);
    if (p && ((uintptr_t)p & 255u)) {  // unaligned: the vector loads would fault
      s->alloc.free(p, bytes, (void*)s->stream, s->alloc.user);
      p = nullptr;
    }
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) list.push_back({p, bytes});
  return p;
}

void ns_free(sph_nsearch* s, std::vector<sph_nsearch::Blk>& list) {
  for (auto& b : list) {
    if (s->has_alloc)
      s->alloc.free(b.p, b.b, (void*)s->stream, s->alloc.user);
    else
      cudaFree(b.p);
  }
  list.clear();
}

// Cell index of a float coordinate: the same value as cell_coord_fast on the
// widened coordinate (the plain double formula), with no double arithmetic
// off the faces.  x - lo is formed in float against lo split into
// lo_hi + lo_lo (floats, |lo - lo_hi - lo_lo| <= 2^-48 |lo|); with the product
// by the float 1 / cs that is four float roundings (< 2.4e-7 relative), inside
// the distance the test below asks of the quotient from the nearest integer.
// Nearer a face the double subtraction and division decide.
__device__ __forceinline__ int cell_coord_f32(float x, double lo, float lo_hi, float lo_lo,
                                              double cs, float inv_cs, int nc, int& oob) {
  const float qf = __fmul_rn(__fsub_rn(__fsub_rn(x, lo_hi), lo_lo), inv_cs);
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
  return cell_coord_fast((double)x, lo, cs, inv_cs, nc, oob);
}

template <class T>
__device__ __forceinline__ int ns_cell(T x, const Params& P, int k, float inv_cs, int nc,
                                       int& oob) {
  if constexpr (sizeof(T) == 4) {
    const float lo_hi = (float)P.lo[k];
    const float lo_lo = (float)(P.lo[k] - (double)lo_hi);
    return cell_coord_f32(x, P.lo[k], lo_hi, lo_lo, P.cs, inv_cs, nc, oob);
  } else {
    return cell_coord_fast(x, P.lo[k], P.cs, inv_cs, nc, oob);
  }
}

// Cell key from float or double coordinates, with the same value as the
// simulation path's formula on the coordinate widened to double (clamped;
// this entry point reports no out-of-domain flag).
// Also packs each particle's coordinates into one vector (pk, input order),
// so that the reorder gathers one vector per particle instead of one sector
// per coordinate.
template <class T>
__global__ void k_ns_keys(Params P, const T* __restrict__ x, const T* __restrict__ y,
                          const T* __restrict__ z, int n, uint32_t* keys, uint32_t* vals,
                          uint32_t* digit_total, int bins, typename Vec4<T>::type* pk) {
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < bins; t += blockDim.x) digit_total[t] = 0;
  const float inv_cs = (float)(1.0 / P.cs);
  int oob = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const T xi = x[i], yi = y[i], zi = P.dim == 3 ? z[i] : T(0);
    const int cx = ns_cell<T>(xi, P, 0, inv_cs, P.nx, oob);
    const int cy = ns_cell<T>(yi, P, 1, inv_cs, P.ny, oob);
    const int cz = P.dim == 3 ? ns_cell<T>(zi, P, 2, inv_cs, P.nz, oob) : 0;
    typename Vec4<T>::type v;
    v.x = xi;
    v.y = yi;
    v.z = zi;
    v.w = T(0);
    pk[i] = v;
    keys[i] = ((uint32_t)cz * (uint32_t)P.ny + (uint32_t)cy) * (uint32_t)P.nx + (uint32_t)cx;
    vals[i] = (uint32_t)i;
  }
}

// Sorted positions packed as one vector per particle (x, y, z, 0): the density
// pass then reads each candidate with a single load.  The gather takes the
// packed input (one sector per particle; three 4-byte gathers from the
// coordinate arrays fetched about 240 B of DRAM per particle).
template <class T>
__global__ void k_ns_reorder(const uint32_t* __restrict__ perm,
                             const typename Vec4<T>::type* __restrict__ pk, int n,
                             typename Vec4<T>::type* sp) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    sp[k] = pk[perm[k]];
}

// sigma_i = sum over the 3^d cells of W(r_ij), r < 2h, self included (the
// density-summation pass), arithmetic in the position type.
template <class T, class Slots>
__device__ __forceinline__ void ns_density_slots(const Params& P, const uint32_t* __restrict__ keys,
                                                 const uint32_t* __restrict__ cb,
                                                 const typename Vec4<T>::type* __restrict__ sp,
                                                 double* sigma, const Slots& slots) {
  const T r2max = (T)P.r2max, inv_h = (T)(1.0 / P.h), cw = (T)P.walpha;
  const float m_half_inv_h = (float)(-0.5 / P.h), two_inv_h = (float)(2.0 / P.h);
  slots.each([&](const int i) {
    const uint32_t key = keys[i];
    const uint32_t r = key / (uint32_t)P.nx;
    const int cx = (int)(key - r * (uint32_t)P.nx), cy = (int)(r % (uint32_t)P.ny),
              cz = (int)(r / (uint32_t)P.ny);
    const typename Vec4<T>::type pi = sp[i];
    const T xi = pi.x, yi = pi.y, zi = pi.z;
    T sig = 0;
    const int kz = P.dim == 3 ? 1 : 0;
    for (int dz = -kz; dz <= kz; ++dz) {
      const int zz = cz + dz;
      if (zz < 0 || zz >= P.nz) continue;
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = cy + dy;
        if (yy < 0 || yy >= P.ny) continue;
        const uint32_t row = ((uint32_t)zz * (uint32_t)P.ny + (uint32_t)yy) * (uint32_t)P.nx;
        const uint32_t c0 = row + (uint32_t)(cx > 0 ? cx - 1 : cx);
        const uint32_t c1 = row + (uint32_t)(cx + 1 < P.nx ? cx + 1 : cx);
        const uint32_t e = cb[c1 + 1];
#pragma unroll 4  // measured +1% with the folded constants (-1% without)
        for (uint32_t j = cb[c0]; j < e; ++j) {  // the row's 3 cells are contiguous
          const typename Vec4<T>::type pj = sp[j];
          const T dx = xi - pj.x, dyv = yi - pj.y, dzv = zi - pj.z;
          const T r2 = dx * dx + dyv * dyv + dzv * dzv;
          if (r2 < r2max) {
            if constexpr (sizeof(T) == 4) {
              // W / walpha = t^4 (2q + 1), t = 1 - q/2, q = r / h, with r from
              // the approximate reciprocal square root (relative error about
              // 2^-22; r^2 = 0 gives r = 0) and the constants folded: the
              // accepted branch runs for the warp at nearly every candidate
              float rs;
              asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(r2 + 1e-30f));
              const float r = r2 * rs;
              const float t = fmaf(r, m_half_inv_h, 1.0f);
              const float t2 = t * t;
              sig = fmaf(t2 * t2, fmaf(r, two_inv_h, 1.0f), sig);
            } else {
              const T q = sqrt(r2) * inv_h;
              const T t = T(1) - T(0.5) * q;
              const T t2 = t * t;
              sig += t2 * t2 * (T(2) * q + T(1));
            }
          }
        }
      }
    }
    sigma[i] = (double)(cw * sig);  // the kernel constant once per particle
  });
}

// The slots in brick order (UnitSlots over U's arrays): measured 2.16e9 ->
// 2.68e9 particles/s on the 2^24-particle search against the strided walk.
template <class T>
__global__ void __launch_bounds__(256) k_ns_density(Params P, const uint32_t* __restrict__ keys,
                                                    const uint32_t* __restrict__ cb,
                                                    const typename Vec4<T>::type* __restrict__ sp,
                                                    int n, double* sigma, DevBuffers U) {
  ns_density_slots<T>(P, keys, cb, sp, sigma,
                      stages::UnitSlots{U.units, U.unit_ctr + 2 * U.parts, U.parts,
                                        (n + 31) >> 5, n});
}

int grid_of(int n, int block, int cap) {
  int b = (n + block - 1) / block;
  return b < 1 ? 1 : (b > cap ? cap : b);
}

}  // namespace

extern "C" {

int sph_nsearch_create(const sph_domain* domain, double h, int pos_precision,
                       const sph_allocator* alloc, void* stream, sph_nsearch** out) {
  if (!out || !domain || !(h > 0)) return SPH_E_INVALID;
  *out = nullptr;
  if (domain->dim != 2 && domain->dim != 3) return SPH_E_INVALID;
  if (pos_precision != SPH_FP64 && pos_precision != SPH_MIXED) return SPH_E_INVALID;
  if (alloc && (!alloc->alloc || !alloc->free)) return SPH_E_INVALID;
  sph_nsearch* s = new sph_nsearch();
  Params& P = s->P;
  P.dim = domain->dim;
  P.cs = 2.0 * h;
  P.h = h;
  P.r2max = 4.0 * h * h;
  P.walpha = P.dim == 2 ? 7.0 / (4.0 * kPiN * h * h) : 21.0 / (16.0 * kPiN * h * h * h);
  long long ncell = 1;
  int nc[3] = {1, 1, 1};
  for (int k = 0; k < P.dim; ++k) {
    if (!(domain->hi[k] > domain->lo[k])) {
      delete s;
      return SPH_E_INVALID;
    }
    const long long m = grid_cells(domain->lo[k], domain->hi[k], P.cs);
    if (m < 0) {
      delete s;
      return SPH_E_INVALID;
    }
    nc[k] = (int)m;
    ncell *= m;
    if (ncell > 0xfffffffell) {
      delete s;
      return SPH_E_INVALID;
    }
    P.lo[k] = domain->lo[k];
  }
  if (ncell > 0xfffffffell) {
    delete s;
    return SPH_E_INVALID;
  }
  P.nx = nc[0];
  P.ny = nc[1];
  P.nz = nc[2];
  P.ncell = (uint32_t)ncell;
  s->fp32 = pos_precision == SPH_MIXED;
  if (alloc) {
    s->alloc = *alloc;
    s->has_alloc = true;
  }
  s->user_stream = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&s->L.sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  for (int k = 0; k < 6 && e == cudaSuccess; ++k) e = cudaEventCreate(&s->ev[k]);
  if (e == cudaSuccess) e = configure_sort_kernels();
  if (e != cudaSuccess) {
    sph_nsearch_destroy(s);
    return SPH_E_CUDA;
  }
  s->L.block_stream = 256;
  s->L.blocks_stream = s->L.sms * 8;
  s->L.radix_bits = 8;
  s->L.hist_ballot = 1;  // positions in any order: the keys are not nearly sorted
  s->L.key_bits = bits_for(P.ncell);
  s->L.radix_passes = radix_passes_for(s->L.key_bits, s->L.radix_bits);
  s->cell_begin = (uint32_t*)ns_alloc(s, ((size_t)P.ncell + 1) * 4, s->fixed);
  s->digit_total = (uint32_t*)ns_alloc(s, ((size_t)1 << kMaxRadixBits) * 4, s->fixed);
  s->L.block_loop = 128;
  const size_t nb = (size_t)brick_count(P);
  s->U.brick_start = (uint32_t*)ns_alloc(s, (nb + 1) * 4, s->fixed);
  s->U.brick_fill = (uint32_t*)ns_alloc(s, nb * 4, s->fixed);
  s->U.unit_ctr = (uint32_t*)ns_alloc(s, 5 * (size_t)s->L.sms * 4, s->fixed);
  s->U.parts = s->L.sms;
  if (!s->cell_begin || !s->digit_total || !s->U.brick_start || !s->U.brick_fill ||
      !s->U.unit_ctr) {
    sph_nsearch_destroy(s);
    return SPH_E_OOM;
  }
  *out = s;
  return SPH_OK;
}

int sph_nsearch_run(sph_nsearch* s, size_t n, const void* x, const void* y, const void* z,
                    double* stage_ms) {
  if (!s || n == 0 || n >= (1ull << 31) || !x || !y || (s->P.dim == 3 && !z))
    return SPH_E_INVALID;
  const size_t ts = s->fp32 ? 4 : 8;
  if (n > s->cap) {
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return SPH_E_CUDA;
    ns_free(s, s->blocks);
    bool ok = true;
    for (int p = 0; p < 2; ++p) {
      s->keys[p] = (uint32_t*)ns_alloc(s, n * 4, s->blocks);
      s->vals[p] = (uint32_t*)ns_alloc(s, n * 4, s->blocks);
      ok &= s->keys[p] && s->vals[p];
    }
    s->sp = ns_alloc(s, n * 4 * ts, s->blocks);
    s->pk = ns_alloc(s, n * 4 * ts, s->blocks);
    ok &= s->sp != nullptr && s->pk != nullptr;
    s->sigma = (double*)ns_alloc(s, n * 8, s->blocks);
    s->U.units = (uint32_t*)ns_alloc(s, ((n + 31) / 32) * 4, s->blocks);
    s->U.unit_brick = (uint32_t*)ns_alloc(s, ((n + 31) / 32) * 4, s->blocks);
    ok &= s->U.units && s->U.unit_brick;
    const size_t tiles = (n + kSortTile - 1) / kSortTile;
    s->tile_hist = (uint32_t*)ns_alloc(s, tiles * ((size_t)1 << kMaxRadixBits) * 4, s->blocks);
    ok &= s->sigma && s->tile_hist;
    if (!ok) {
      ns_free(s, s->blocks);
      s->cap = 0;
      return SPH_E_OOM;
    }
    s->cap = n;
  }
  s->n = n;
  s->P.n = (int)n;
  cudaStream_t st = s->stream;
  if (cudaEventRecord(s->ev[0], s->user_stream) != cudaSuccess) return SPH_E_CUDA;
  if (cudaStreamWaitEvent(st, s->ev[0], 0) != cudaSuccess) return SPH_E_CUDA;
  const int ni = (int)n;
  const int gs = grid_of(ni, 256, s->L.blocks_stream);
  const int bins = 1 << s->L.radix_bits;
  cudaEventRecord(s->ev[0], st);
  if (s->fp32)
    k_ns_keys<float><<<gs, 256, 0, st>>>(s->P, (const float*)x, (const float*)y, (const float*)z,
                                         ni, s->keys[0], s->vals[0], s->digit_total, bins,
                                         (float4*)s->pk);
  else
    k_ns_keys<double><<<gs, 256, 0, st>>>(s->P, (const double*)x, (const double*)y,
                                          (const double*)z, ni, s->keys[0], s->vals[0],
                                          s->digit_total, bins, (double4_32a*)s->pk);
  cudaEventRecord(s->ev[1], st);
  s->sorted = launch_radix_sort(s->L, s->keys, s->vals, ni, s->tile_hist, s->digit_total,
                                nullptr, 0, st);
  cudaEventRecord(s->ev[2], st);
  const uint32_t* perm = s->vals[s->sorted];
  const uint32_t* keys = s->keys[s->sorted];
  if (s->fp32)
    k_ns_reorder<float><<<gs, 256, 0, st>>>(perm, (const float4*)s->pk, ni, (float4*)s->sp);
  else
    k_ns_reorder<double><<<gs, 256, 0, st>>>(perm, (const double4_32a*)s->pk, ni,
                                             (double4_32a*)s->sp);
  cudaEventRecord(s->ev[3], st);
  launch_cell_offsets(keys, ni, s->P.ncell, s->cell_begin, nullptr, 0, 0, st);
  cudaEventRecord(s->ev[4], st);
  // density pass in brick order: the sorted keys' 32-slot groups by brick,
  // then one resident wave claiming them (counted in the density stage)
  DevBuffers U = s->U;
  U.binned = keys;
  {
    const int ng = (ni + 31) >> 5;
    const int gu = grid_of(ng, 256, s->L.blocks_stream);
    const int nclear = (int)brick_count(s->P) + 1 > 3 * U.parts ? (int)brick_count(s->P) + 1
                                                                 : 3 * U.parts;
    stages::k_units_clear<3><<<grid_of(nclear, 256, s->L.blocks_stream), 256, 0, st>>>(s->P, U, 0);
    stages::k_units_count<3><<<gu, 256, 0, st>>>(s->P, U, 0);
    stages::k_units_scan<3><<<1, stages::kUnitScanThreads, 0, st>>>(s->P, U, 0);
    stages::k_units_scatter<3><<<gu, 256, 0, st>>>(s->P, U, 0);
  }
  if (s->fp32)
    k_ns_density<float><<<stages::one_wave(k_ns_density<float>, s->L), 128, 0, st>>>(
        s->P, keys, s->cell_begin, (const float4*)s->sp, ni, s->sigma, U);
  else
    k_ns_density<double><<<stages::one_wave(k_ns_density<double>, s->L), 128, 0, st>>>(
        s->P, keys, s->cell_begin, (const double4_32a*)s->sp, ni, s->sigma, U);
  cudaEventRecord(s->ev[5], st);
  if (cudaGetLastError() != cudaSuccess) return SPH_E_CUDA;
  if (stage_ms) {
    if (cudaEventSynchronize(s->ev[5]) != cudaSuccess) return SPH_E_CUDA;
    for (int k = 0; k < 5; ++k) {
      float t = 0.f;
      cudaEventElapsedTime(&t, s->ev[k], s->ev[k + 1]);
      stage_ms[k] = t;
    }
  }
  if (cudaEventRecord(s->ev[0], st) != cudaSuccess) return SPH_E_CUDA;
  return cudaStreamWaitEvent(s->user_stream, s->ev[0], 0) == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}

int sph_nsearch_results(sph_nsearch* s, uint32_t* keys, uint32_t* perm, uint32_t* cell_begin,
                        double* sigma) {
  if (!s || !s->n) return SPH_E_STATE;
  cudaStream_t st = s->stream;
  const size_t n = s->n;
  cudaError_t e = cudaSuccess;
  if (keys) e = cudaMemcpyAsync(keys, s->keys[s->sorted], n * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && perm)
    e = cudaMemcpyAsync(perm, s->vals[s->sorted], n * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && cell_begin)
    e = cudaMemcpyAsync(cell_begin, s->cell_begin, ((size_t)s->P.ncell + 1) * 4,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && sigma) e = cudaMemcpyAsync(sigma, s->sigma, n * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}

size_t sph_nsearch_cell_count(const sph_nsearch* s) { return s ? (size_t)s->P.ncell : 0; }

void sph_nsearch_destroy(sph_nsearch* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  ns_free(s, s->blocks);
  ns_free(s, s->fixed);
  for (int k = 0; k < 6; ++k)
    if (s->ev[k]) cudaEventDestroy(s->ev[k]);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
