// Host-side helpers shared by the context types of the C ABI: device memory
// through the caller's allocator (or cudaMalloc), and the reference number
// density of the particle lattice.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sph.h"

namespace sphgb {

// Host trace range over one public call (NVTX: shows up in nsys / ncu
// timelines under the call's name; free when no tool is attached).
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

struct Block {
  void* p;
  size_t bytes;
};

// Allocations of one object, all on its stream.
struct DevMem {
  sph_allocator alloc{};
  bool has_alloc = false;
  cudaStream_t stream = nullptr;

  void* get(size_t bytes, std::vector<Block>& list) const {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (has_alloc) {
      p = alloc.alloc(bytes, (void*)stream, alloc.user);
      if (p && ((uintptr_t)p & 255u)) {  // unaligned: the vector loads would fault
        alloc.free(p, bytes, (void*)stream, alloc.user);
        p = nullptr;
      }
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) list.push_back({p, bytes});
    return p;
  }
  void release(std::vector<Block>& list) const {
    for (auto& b : list) {
      if (has_alloc)
        alloc.free(b.p, b.bytes, (void*)stream, alloc.user);
      else
        cudaFree(b.p);
    }
    list.clear();
  }
};

// Device copy of every allocation of an object, so that trial runs (the
// autotuner) leave the object exactly as they found it.
struct Snapshot {
  std::vector<Block> src, saved;

  bool take(const DevMem& mem, const std::vector<const std::vector<Block>*>& lists) {
    for (auto* l : lists)
      for (auto& b : *l) src.push_back(b);
    for (auto& b : src)
      if (!mem.get(b.bytes, saved)) {
        drop(mem);
        return false;
      }
    return copy(true, mem.stream) == cudaSuccess;
  }
  cudaError_t copy(bool save, cudaStream_t s) const {
    for (size_t k = 0; k < src.size(); ++k) {
      cudaError_t e = save ? cudaMemcpyAsync(saved[k].p, src[k].p, src[k].bytes,
                                             cudaMemcpyDeviceToDevice, s)
                           : cudaMemcpyAsync(src[k].p, saved[k].p, src[k].bytes,
                                             cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  cudaError_t restore(cudaStream_t s) const { return copy(false, s); }
  void drop(const DevMem& mem) {
    mem.release(saved);
    src.clear();
  }
};

// Coordinate search of the launch configuration: first the block size (the
// tile of a batch), then the radix width of the sort, then neighbour lists on
// or off, each time keeping the fastest.  trial(cfg) restores the object,
// applies cfg and returns its time per acoustic step in ms (< 0: error, which
// ends the search).  Every configuration computes the same results; only the
// time differs.
template <class Trial>
int tune_search(sph_tuning start, Trial trial, sph_tuning* best) {
  sph_tuning b = start;
  int trials = 0;
  double ms = trial(b);
  ++trials;
  if (ms < 0) return -1;
  b.ms_per_step = ms;
  const int blocks[] = {64, 96, 128, 192, 256};
  const int block0 = b.block;
  for (int v : blocks) {
    if (v == block0) continue;
    sph_tuning c = b;
    c.block = v;
    const double t = trial(c);
    ++trials;
    if (t < 0) return -1;
    if (t < b.ms_per_step) {
      b = c;
      b.ms_per_step = t;
    }
  }
  const int radix0 = b.radix_bits;
  for (int v = 5; v <= 11; ++v) {
    if (v == radix0) continue;
    sph_tuning c = b;
    c.radix_bits = v;
    const double t = trial(c);
    ++trials;
    if (t < 0) return -1;
    if (t < b.ms_per_step) {
      b = c;
      b.ms_per_step = t;
    }
  }
  {
    sph_tuning c = b;
    c.neighbour_list = !b.neighbour_list;
    const double t = trial(c);
    ++trials;
    if (t < 0) return -1;
    if (t < b.ms_per_step) {
      b = c;
      b.ms_per_step = t;
    }
  }
  b.trials = trials;
  *best = b;
  return 0;
}

constexpr double kPiHost = 3.14159265358979323846;

inline double wendland_alpha(int dim, double h) {
  return dim == 2 ? 7.0 / (4.0 * kPiHost * h * h) : 21.0 / (16.0 * kPiHost * h * h * h);
}

// Reference number density sigma0: the kernel summed over the unperturbed
// lattice of spacing dp around one particle (self included).
inline double lattice_sigma0(int dim, double dp, double h, double walpha) {
  const int K = (int)std::ceil(2.0 * h / dp) + 1;
  const int kz = dim == 3 ? K : 0;
  double s = 0.0;
  for (int c = -kz; c <= kz; ++c)
    for (int b = -K; b <= K; ++b)
      for (int a = -K; a <= K; ++a) {
        const double r = dp * std::sqrt((double)(a * a + b * b + c * c));
        const double q = r / h;
        if (q >= 2.0) continue;
        const double t = 1.0 - 0.5 * q;
        s += walpha * t * t * t * t * (2.0 * q + 1.0);
      }
  return s;
}

}  // namespace sphgb
