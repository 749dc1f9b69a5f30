// Cell sort that allocates nothing: the radix sort's scratch lives in a
// file-scope device array instead of memory obtained at run time.
//
// Some callers cannot allocate device memory when they need the sort: code
// that runs with a fixed memory budget handed out up front, code that must not
// stall (cudaMalloc and cudaFree synchronise the device), or code that runs
// where no allocator is reachable.  This entry point serves them.  The array
// is sized for SPH_NOALLOC_MAX_PARTICLES particles and is held by every GPU
// that loads the library until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>

#include "sph.h"
#include "sph_internal.cuh"

using namespace sphgb;

namespace {

constexpr size_t kMaxN = SPH_NOALLOC_MAX_PARTICLES;
constexpr int kRadixBits = 8;
constexpr size_t kBins = (size_t)1 << kRadixBits;
constexpr size_t kMaxTiles = (kMaxN + kSortTile - 1) / kSortTile;
// keys and values of one ping-pong side, per-tile histograms, digit totals
constexpr size_t kScratchWords = 2 * kMaxN + kMaxTiles * kBins + kBins;

static __device__ __align__(256) uint32_t g_sort_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint32_t* g_scratch[kMaxDevices];  // device address of g_sort_scratch, per device
int g_sms[kMaxDevices];
bool g_ready[kMaxDevices];

// One-time set-up for the current device: the device address of the array
// (host code may not use the symbol itself as an address), the shared-memory
// limits of the sort kernels, and the multiprocessor count.
int setup_current_device(int dev) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_ready[dev]) return SPH_OK;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || !p) return SPH_E_CUDA;
  if (configure_sort_kernels() != cudaSuccess) return SPH_E_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SPH_E_CUDA;
  g_scratch[dev] = (uint32_t*)p;
  g_sms[dev] = sms;
  g_ready[dev] = true;
  return SPH_OK;
}

}  // namespace

extern "C" int sph_cell_sort_noalloc(const sph_domain* domain, double cell_size, const double* x,
                                     const double* y, const double* z, size_t n,
                                     uint32_t* keys_out, uint32_t* perm_out,
                                     uint32_t* cell_begin_out, void* stream) {
  if (!domain || !(cell_size > 0) || !keys_out || !perm_out || !cell_begin_out)
    return SPH_E_INVALID;
  const int dim = domain->dim;
  if (dim != 2 && dim != 3) return SPH_E_INVALID;
  if (n > kMaxN) return SPH_E_INVALID;  // beyond the static scratch
  if (n > 0 && (!x || !y || (dim == 3 && !z))) return SPH_E_INVALID;
  Params P{};
  P.dim = dim;
  long long ncell = 1;
  int nc[3] = {1, 1, 1};
  for (int k = 0; k < dim; ++k) {
    if (!(domain->hi[k] > domain->lo[k])) return SPH_E_INVALID;
    const long long m = grid_cells(domain->lo[k], domain->hi[k], cell_size);
    if (m < 0) return SPH_E_INVALID;
    nc[k] = (int)m;
    ncell *= m;
    if (ncell > 0xfffffffell) return SPH_E_INVALID;
    P.lo[k] = domain->lo[k];
  }
  P.nx = nc[0];
  P.ny = nc[1];
  P.nz = nc[2];
  P.ncell = (uint32_t)ncell;
  P.cs = cell_size;
  P.n = (int)n;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SPH_E_CUDA;
  int rc = setup_current_device(dev);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  LaunchCfg L{};
  L.sms = g_sms[dev];
  L.block_stream = 256;
  L.blocks_stream = L.sms * 8;
  L.radix_bits = kRadixBits;
  L.key_bits = bits_for(P.ncell);
  L.radix_passes = radix_passes_for(L.key_bits, L.radix_bits);

  uint32_t* base = g_scratch[dev];
  uint32_t* sk = base;
  uint32_t* sv = base + kMaxN;
  uint32_t* tile_hist = base + 2 * kMaxN;
  uint32_t* digit_total = tile_hist + kMaxTiles * kBins;
  // place the ping-pong so that the last pass writes the caller's arrays
  const bool odd = L.radix_passes % 2 == 1;
  uint32_t* keys[2] = {odd ? sk : keys_out, odd ? keys_out : sk};
  uint32_t* vals[2] = {odd ? sv : perm_out, odd ? perm_out : sv};

  if (n > 0) {
    const double* xs[3] = {x, y, dim == 3 ? z : x};
    // the key kernel also clears the digit totals left by the previous call
    launch_cell_keys(P, L, xs, keys[0], vals[0], (int)n, nullptr, 0, digit_total, s);
    launch_radix_sort(L, keys, vals, (int)n, tile_hist, digit_total, nullptr, 0, s);
  }
  launch_cell_offsets(keys_out, (int)n, P.ncell, cell_begin_out, nullptr, 0, 0, s);
  return cudaGetLastError() == cudaSuccess ? SPH_OK : SPH_E_CUDA;
}
