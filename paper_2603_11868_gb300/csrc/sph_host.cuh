// Host-side helpers shared by the context types of the C ABI: device memory
// through the caller's allocator (or cudaMalloc), and the reference number
// density of the particle lattice.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "sph.h"

namespace sphgb {

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
