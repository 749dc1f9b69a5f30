// C ABI of the GB300 SPH library (declared in include/sph.h): context
// management, device memory through the caller's allocator, stream ordering
// with the caller's stream, CUDA-graph replay of the acoustic step, and field
// transfer in user order.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cstddef>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <string>
#include <thread>
#include <vector>

#include "sph.h"
#include "sph_host.cuh"
#include "sph_internal.cuh"

using namespace sphgb;

struct sph_ctx {
  Params P{};
  LaunchCfg L{};
  DevBuffers B{};
  int precision = SPH_MIXED;
  sph_allocator alloc{};
  bool has_alloc = false;
  cudaStream_t user_stream = nullptr;
  cudaStream_t stream = nullptr;  // internal, non-blocking
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  bool use_graph = true;
  int device = 0;
  double dp = 0;
  size_t cap_n = 0;   // capacity of per-particle buffers
  size_t cap_nw = 0;  // capacity of wall buffers
  // trans_blocks: the buffers of translating walls (sph_set_wall_translation)
  std::vector<Block> fluid_blocks, wall_blocks, fixed_blocks, trans_blocks;
  std::vector<double> wall_vel_host;  // given wall velocities (n * dim), empty at rest
  bool motion_owns_vel = false;  // wall velocity arrays allocated by sph_set_wall_motion
  std::string err;
  bool fluid_set = false;
};

namespace {

double __longlong_as_double_host(long long v) {
  double d;
  memcpy(&d, &v, sizeof d);
  return d;
}
long long __double_as_longlong_host(double d) {
  long long v;
  memcpy(&v, &d, sizeof v);
  return v;
}

int set_err(sph_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_err(sph_ctx* c, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return SPH_OK;
  return set_err(c, SPH_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// The neighbour lists name walls by their sorted slot: once the walls are
// sorted anew outside a rebuild, the loops take direct search until the next
// rebuild builds fresh lists.
cudaError_t invalidate_lists(sph_ctx* c) {
  const int one = 1;
  return cudaMemcpyAsync((char*)c->B.sc + offsetof(DevScalars, list_bad), &one, sizeof(int),
                         cudaMemcpyHostToDevice, c->stream);
}

// forgets the translating walls (their buffers are freed by the caller)
void clear_translation(sph_ctx* c) {
  c->B.wall_moves = nullptr;
  c->B.wall_io = nullptr;
  c->B.wall_key = nullptr;
  c->B.wkeys[0] = c->B.wkeys[1] = nullptr;
  c->B.wvals[0] = c->B.wvals[1] = nullptr;
  c->B.wtile_hist = nullptr;
  c->B.wall_amp = nullptr;
  c->B.wall_acc = nullptr;
  c->P.variant &= ~(kVariantTranslatingWall | kVariantAccelWall);
  c->P.wall_vmax = 0.0;
  c->P.wall_omega = 0.0;
  if (c->motion_owns_vel) {
    c->B.wall_vel = nullptr;
    c->B.wall_v0 = nullptr;
    c->P.variant &= ~kVariantMovingWall;
    c->motion_owns_vel = false;
  }
}

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_err(c, e_, #call); \
  } while (0)

void* dev_alloc(sph_ctx* c, size_t bytes, std::vector<Block>& list) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~(size_t)255;
  void* p = nullptr;
  if (c->has_alloc) {
    p = c->alloc.alloc(bytes, (void*)c->stream, c->alloc.user);
    if (p && ((uintptr_t)p & 255u)) {  // unaligned: the vector loads would fault
      c->alloc.free(p, bytes, (void*)c->stream, c->alloc.user);
      p = nullptr;
    }
  } else {
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  if (p) list.push_back({p, bytes});
  return p;
}

void dev_free_list(sph_ctx* c, std::vector<Block>& list) {
  for (auto& b : list) {
    if (c->has_alloc)
      c->alloc.free(b.p, b.bytes, (void*)c->stream, c->alloc.user);
    else
      cudaFree(b.p);
  }
  list.clear();
}

void drop_graph(sph_ctx* c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->graph_exec = nullptr;
  c->graph = nullptr;
}

size_t tsize(const sph_ctx* c) { return c->precision == SPH_FP64 ? 8 : 4; }

StageArgs args(const sph_ctx* c) {
  StageArgs a;
  a.P = c->P;
  a.B = c->B;
  a.B.binned = a.B.keys[a.B.sorted_buf];
  a.L = c->L;
  return a;
}

void enqueue_step(sph_ctx* c, cudaStream_t s) {
  if (c->precision == SPH_FP64)
    enqueue_step_fp64(args(c), s);
  else
    enqueue_step_mixed(args(c), s);
}

// The acoustic step as a CUDA graph: the schedule kernel, then a conditional
// node holding the stages of a step that begins an advection step (cell keys,
// sort, reorder, offsets, lists, density summation, viscous force), then the
// acoustic stages.  The schedule kernel sets the condition on the device, so a
// step inside an advection step launches four kernels instead of the rebuild
// chain of early-exiting ones.
cudaError_t capture_step_graph(sph_ctx* c, cudaGraph_t* out) {
  *out = nullptr;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle cond;
  // the condition starts every launch at 0 (skip) until the schedule sets it
  e = cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault);
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(c->stream, g, nullptr, nullptr, 0, mode);
  if (e == cudaSuccess) {
    launch_control_cond(c->P, c->B.sc, cond, c->stream);
    e = cudaStreamEndCapture(c->stream, &g);
  }
  cudaGraphNode_t control = nullptr;
  size_t count = 1;
  if (e == cudaSuccess) e = cudaGraphGetNodes(g, &control, &count);
  if (e == cudaSuccess && count != 1) e = cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeIf;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, g, &control, nullptr, 1, &cp);
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0, mode);
    if (e == cudaSuccess) {
      if (c->precision == SPH_FP64)
        enqueue_advection_fp64(args(c), c->stream);
      else
        enqueue_advection_mixed(args(c), c->stream);
      e = cudaStreamEndCapture(c->stream, &body);
    }
  }
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(c->stream, g, &cnode, nullptr, 1, mode);
  if (e == cudaSuccess) {
    if (c->precision == SPH_FP64)
      enqueue_acoustic_fp64(args(c), c->stream);
    else
      enqueue_acoustic_mixed(args(c), c->stream);
    e = cudaStreamEndCapture(c->stream, &g);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return e;
  }
  *out = g;
  return cudaSuccess;
}

void configure_launch(sph_ctx* c) {
  LaunchCfg& L = c->L;
  if (L.block_loop <= 0) L.block_loop = 128;
  L.blocks_loop = L.sms * (2048 / L.block_loop);
  L.block_stream = 256;
  L.blocks_stream = L.sms * 8;
  L.key_bits = bits_for(c->P.ncell);
  L.radix_passes = radix_passes_for(L.key_bits, L.radix_bits);
  c->B.sorted_buf = L.radix_passes % 2;
}

// The caller's stream -> internal stream ordering.
int enter(sph_ctx* c) {
  CK(cudaEventRecord(c->ev_in, c->user_stream));
  CK(cudaStreamWaitEvent(c->stream, c->ev_in, 0));
  return SPH_OK;
}
int leave(sph_ctx* c) {
  CK(cudaEventRecord(c->ev_out, c->stream));
  CK(cudaStreamWaitEvent(c->user_stream, c->ev_out, 0));
  return SPH_OK;
}

int read_scalars(sph_ctx* c, DevScalars* hs) {
  CK(cudaMemcpyAsync(hs, c->B.sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SPH_OK;
}

int flags_status(sph_ctx* c, const DevScalars& hs) {
  if (hs.flags & kFlagIndex)
    return set_err(c, SPH_E_INDEX, "an index check of the debug build failed");
  if (hs.flags & kFlagNonFinite)
    return set_err(c, SPH_E_NONFINITE, "a velocity or density became non-finite");
  if (hs.flags & kFlagOutOfDomain)
    return set_err(c, SPH_E_OUT_OF_DOMAIN, "a particle left the domain (clamped to the edge cell)");
  return SPH_OK;
}

int sync_status(sph_ctx* c, DevScalars* out = nullptr) {
  DevScalars hs;
  int rc = read_scalars(c, &hs);
  if (rc) return rc;
  CK(cudaGetLastError());
  if (out) *out = hs;
  return flags_status(c, hs);
}

// user-order scatter of one field: out[id[k] * comps + q] = src_q[k * stride + off]
__global__ void k_iota(uint32_t* a, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = i;
}

__global__ void k_scatter_field(const void* s0, const void* s1, const void* s2, int is_float,
                                int stride, int off, int comps, const uint32_t* __restrict__ id,
                                int n, double* __restrict__ out) {
  const void* src[3] = {s0, s1, s2};
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const size_t u = id[k];
    for (int q = 0; q < comps; ++q) {
      const size_t e = (size_t)k * stride + off;
      out[u * comps + q] = is_float ? (double)((const float*)src[q])[e] : ((const double*)src[q])[e];
    }
  }
}

int scatter_out(sph_ctx* c, const void* s0, const void* s1, const void* s2, int is_float,
                int stride, int off, int comps, int par, double* host) {
  const int n = c->P.n;
  int blocks = (n + 255) / 256;
  if (blocks > c->L.blocks_stream) blocks = c->L.blocks_stream;
  if (blocks < 1) blocks = 1;
  k_scatter_field<<<blocks, 256, 0, c->stream>>>(s0, s1, s2, is_float, stride, off, comps,
                                                 c->B.id[par], n, c->B.io);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(host, c->B.io, (size_t)n * comps * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return SPH_OK;
}

int alloc_fluid(sph_ctx* c, size_t n) {
  if (n <= c->cap_n && !c->fluid_blocks.empty()) return SPH_OK;
  CK(cudaStreamSynchronize(c->stream));
  drop_graph(c);
  dev_free_list(c, c->fluid_blocks);
  DevBuffers& B = c->B;
  const size_t ts = tsize(c);
  const int d = c->P.dim;
  const size_t nn = n ? n : 1;
  auto A = [&](size_t bytes) { return dev_alloc(c, bytes, c->fluid_blocks); };
  bool ok = true;
  for (int p = 0; p < 2; ++p) {
    for (int k = 0; k < 3; ++k) {
      B.x[p][k] = k < d ? (double*)A(nn * 8) : nullptr;
      B.v[p][k] = k < d ? (double*)A(nn * 8) : nullptr;
      ok &= k >= d || (B.x[p][k] && B.v[p][k]);
    }
    B.rho[p] = (double*)A(nn * 8);
    B.drho[p] = A(nn * ts);
    B.id[p] = (uint32_t*)A(nn * 4);
    ok &= B.rho[p] && B.drho[p] && B.id[p];
  }
  for (int k = 0; k < 3; ++k) {
    B.aprior[k] = k < d ? A(nn * ts) : nullptr;
    B.acc[k] = k < d ? A(nn * ts) : nullptr;
    ok &= k >= d || (B.aprior[k] && B.acc[k]);
  }
  B.sigma = A(nn * ts);
  B.sigma64 = (double*)A(nn * 8);
  for (int k = 0; k < 3; ++k) {
    B.xreb[k] = k < d ? A(nn * ts) : nullptr;
    ok &= k >= d || B.xreb[k];
  }
  B.bud = (float*)A(nn * 4);
  B.brec = A(nn * 4 * ts);
  ok &= B.bud != nullptr && B.brec != nullptr;
  ok &= B.sigma64 != nullptr;
  for (int p = 0; p < 2; ++p) {
    B.rec[p] = A(nn * (d == 3 ? 8 : 4) * ts);
    B.rec_s[p] = d == 3 ? nullptr : A(nn * 2 * ts);
    B.keys[p] = (uint32_t*)A(nn * 4);
    B.vals[p] = (uint32_t*)A(nn * 4);
    ok &= B.rec[p] && (d == 3 || B.rec_s[p]) && B.keys[p] && B.vals[p];
  }
  B.recI = c->precision == SPH_MIXED ? A(nn * (d == 3 ? 16 : 8)) : nullptr;
  ok &= c->precision != SPH_MIXED || B.recI;
  // neighbour lists: capacity entries per particle, whole warps of 32
  const size_t warps = (nn + 31) / 32;
  // two extra rows of 32 entries: the list walk reads up to two entries past
  // a particle's last one (prefetch), which stays inside the allocation
  B.nl = (uint32_t*)A((warps * (size_t)c->P.list_cap + 2) * 32 * 4);
  if (B.parts) {
    B.units = (uint32_t*)A(warps * 4);
    B.unit_brick = (uint32_t*)A(warps * 4);
    ok &= B.units && B.unit_brick;
    // a valid order (identity) until the first rebuild makes the brick order
    if (B.units) {
      k_iota<<<(int)((warps + 255) / 256), 256, 0, c->stream>>>(B.units, (uint32_t)warps);
      CK(cudaGetLastError());
    }
  }
  B.nl_cnt = (uint32_t*)A(nn * 4);
  ok &= B.nl && B.nl_cnt;
  const size_t tiles = (nn + kSortTile - 1) / kSortTile;
  B.tile_hist = (uint32_t*)A(tiles * ((size_t)1 << kMaxRadixBits) * 4);
  B.io = (double*)A(nn * 3 * 8);
  ok &= B.sigma && B.tile_hist && B.io;
  if (!ok) {
    dev_free_list(c, c->fluid_blocks);
    c->cap_n = 0;
    return set_err(c, SPH_E_OOM, "device allocation failed (fluid buffers)");
  }
  c->cap_n = n;
  return SPH_OK;
}

}  // namespace

extern "C" {

int sph_create(const sph_domain* domain, double dp, double h, const sph_material* mat,
               const double gravity[3], int precision, const sph_allocator* alloc, void* stream,
               sph_ctx** out) {
  if (!out) return SPH_E_INVALID;
  *out = nullptr;
  if (!domain || !mat || !gravity) return SPH_E_INVALID;
  const int dim = domain->dim;
  if (dim != 2 && dim != 3) return SPH_E_INVALID;
  if (!(dp > 0) || !(h > 0) || !(mat->rho0 > 0) || !(mat->c0 > 0) || !(mat->mu >= 0) ||
      !(mat->U_ref > 0))
    return SPH_E_INVALID;
  if (precision != SPH_FP64 && precision != SPH_MIXED) return SPH_E_INVALID;
  if (alloc && (!alloc->alloc || !alloc->free)) return SPH_E_INVALID;
  const double cs = 2.0 * h;
  long long nc[3] = {1, 1, 1};
  long long ncell = 1;
  for (int k = 0; k < dim; ++k) {
    if (!(domain->hi[k] > domain->lo[k])) return SPH_E_INVALID;
    nc[k] = grid_cells(domain->lo[k], domain->hi[k], cs);
    if (nc[k] < 0) return SPH_E_INVALID;
    ncell *= nc[k];
    if (ncell > 0xfffffffell) return SPH_E_INVALID;
  }
  sph_ctx* c = new sph_ctx();
  c->precision = precision;
  c->dp = dp;
  if (alloc) {
    c->alloc = *alloc;
    c->has_alloc = true;
  }
  c->user_stream = (cudaStream_t)stream;
  Params& P = c->P;
  P.dim = dim;
  P.nx = (int)nc[0];
  P.ny = (int)nc[1];
  P.nz = (int)nc[2];
  P.ncell = (uint32_t)ncell;
  for (int k = 0; k < 3; ++k) {
    P.lo[k] = k < dim ? domain->lo[k] : 0.0;
    P.g[k] = k < dim ? gravity[k] : 0.0;
  }
  P.cs = cs;
  P.h = h;
  P.r2max = 4.0 * h * h;
  P.rho0 = mat->rho0;
  P.c0 = mat->c0;
  P.c0sq = mat->c0 * mat->c0;
  P.mu = mat->mu;
  P.U_ref = mat->U_ref;
  P.V = dim == 2 ? dp * dp : dp * dp * dp;
  P.m = mat->rho0 * P.V;
  P.walpha = wendland_alpha(dim, h);
  P.sigma0 = lattice_sigma0(dim, dp, h, P.walpha);
  P.eps = 0.01 * h;
  P.diag = 0;
  P.use_list = 1;
  P.list_cap = dim == 3 ? 192 : 64;
  P.skin_max = 0.6 * h;
  P.variant = 0;

  int rc = SPH_OK;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->L.sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = configure_sort_kernels();
  if (e != cudaSuccess) {
    rc = cuda_err(c, e, "sph_create");
    sph_destroy(c);
    return rc;
  }
  c->L.radix_bits = 8;
  c->L.block_loop = 128;
  configure_launch(c);
  // fixed buffers: scalars and the two CSR offset arrays
  c->B.sc = (DevScalars*)dev_alloc(c, sizeof(DevScalars), c->fixed_blocks);
  c->B.dbg_flags = c->B.sc ? (int*)((char*)c->B.sc + offsetof(DevScalars, flags)) : nullptr;
  c->B.cell_begin = (uint32_t*)dev_alloc(c, ((size_t)P.ncell + 1) * 4, c->fixed_blocks);
  c->B.wall_cb = (uint32_t*)dev_alloc(c, ((size_t)P.ncell + 1) * 4, c->fixed_blocks);
  c->B.digit_total = (uint32_t*)dev_alloc(c, ((size_t)1 << kMaxRadixBits) * 4, c->fixed_blocks);
  c->B.u64_io = (unsigned long long*)dev_alloc(c, 8, c->fixed_blocks);
  if (P.dim == 3 && precision == SPH_MIXED) {
    const size_t nb = (size_t)brick_count(P);
    c->B.brick_start = (uint32_t*)dev_alloc(c, (nb + 1) * 4, c->fixed_blocks);
    c->B.brick_fill = (uint32_t*)dev_alloc(c, nb * 4, c->fixed_blocks);
    c->B.unit_ctr = (uint32_t*)dev_alloc(c, 5 * (size_t)c->L.sms * 4, c->fixed_blocks);
    c->B.parts = c->L.sms;
  }
  double* ctab = nullptr;
  if (precision == SPH_MIXED)
    ctab = (double*)dev_alloc(c, (size_t)(P.nx + P.ny + P.nz) * 8, c->fixed_blocks);
  c->B.ctab = ctab;
  if (!c->B.sc || !c->B.cell_begin || !c->B.wall_cb || !c->B.digit_total || !c->B.u64_io ||
      (precision == SPH_MIXED && !ctab) ||
      (c->B.parts && (!c->B.brick_start || !c->B.brick_fill || !c->B.unit_ctr))) {
    sph_destroy(c);
    return SPH_E_OOM;
  }
  DevScalars z{};
  e = cudaMemcpyAsync(c->B.sc, &z, sizeof(z), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->B.wall_cb, 0, ((size_t)P.ncell + 1) * 4, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->B.digit_total, 0, ((size_t)1 << kMaxRadixBits) * 4, c->stream);
  if (e == cudaSuccess && ctab) {
    launch_centre_table(P, ctab, c->stream);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    rc = cuda_err(c, e, "sph_create");
    sph_destroy(c);
    return rc;
  }
  *out = c;
  return SPH_OK;
}

int sph_set_particles(sph_ctx* c, int kind, size_t n, const double* pos, const double* vel,
                      const double* rho) {
  TraceRange trace_("sph_set_particles");
  if (!c) return SPH_E_INVALID;
  if (n > 0 && !pos) return set_err(c, SPH_E_INVALID, "pos is NULL");
  if (n >= (1ull << 26)) return set_err(c, SPH_E_INVALID, "at most 2^26 - 1 particles per kind");
  const int d = c->P.dim;
  if (kind == SPH_FLUID) {
    int rc = enter(c);
    if (rc) return rc;
    rc = alloc_fluid(c, n);
    if (rc) return rc;
    drop_graph(c);
    c->P.n = (int)n;
    configure_launch(c);
    DevBuffers& B = c->B;
    if (n > 0) {
      // host AoS -> staging -> SoA on the device (no host-side loops)
      CK(cudaMemcpyAsync(B.io, pos, n * d * 8, cudaMemcpyHostToDevice, c->stream));
      launch_deinterleave(B.io, (int)n, d, B.x[0], c->stream);
      if (vel) {
        CK(cudaMemcpyAsync(B.io, vel, n * d * 8, cudaMemcpyHostToDevice, c->stream));
        launch_deinterleave(B.io, (int)n, d, B.v[0], c->stream);
      } else {
        for (int k = 0; k < d; ++k) CK(cudaMemsetAsync(B.v[0][k], 0, n * 8, c->stream));
      }
      if (rho)
        CK(cudaMemcpyAsync(B.rho[0], rho, n * 8, cudaMemcpyHostToDevice, c->stream));
      launch_init_fluid(B.rho[0], rho ? 0 : 1, c->P.rho0, B.id[0], (int)n, c->stream);
      CK(cudaMemsetAsync(B.drho[0], 0, n * tsize(c), c->stream));
      for (int k = 0; k < d; ++k) {
        CK(cudaMemsetAsync(B.acc[k], 0, n * tsize(c), c->stream));
        CK(cudaMemsetAsync(B.aprior[k], 0, n * tsize(c), c->stream));
      }
      CK(cudaMemsetAsync(B.sigma, 0, n * tsize(c), c->stream));
      CK(cudaGetLastError());
    }
    DevScalars z{};
    CK(cudaMemcpyAsync(B.sc, &z, sizeof(z), cudaMemcpyHostToDevice, c->stream));
    if (n > 0) {
      if (c->precision == SPH_FP64)
        enqueue_initial_sort_fp64(args(c), c->stream);
      else
        enqueue_initial_sort_mixed(args(c), c->stream);
      launch_vmax_reset(c->P, c->L, c->B, c->stream);
    } else {
      CK(cudaMemsetAsync(B.cell_begin, 0, ((size_t)c->P.ncell + 1) * 4, c->stream));
    }
    CK(cudaGetLastError());
    c->fluid_set = n > 0;
    CK(cudaStreamSynchronize(c->stream));
    return leave(c);
  }
  if (kind == SPH_WALL) {
    if (rho) return set_err(c, SPH_E_INVALID, "wall particles take no density");
    // a prescribed (sliding) velocity: the walls read it only if one is nonzero
    bool moving = false;
    if (vel) {
      for (size_t q = 0; q < n * (size_t)d; ++q) {
        if (!std::isfinite(vel[q]))
          return set_err(c, SPH_E_INVALID, "wall velocity is not finite");
        moving = moving || vel[q] != 0.0;
      }
    }
    int rc = enter(c);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    drop_graph(c);
    dev_free_list(c, c->trans_blocks);
    dev_free_list(c, c->wall_blocks);
    clear_translation(c);
    c->cap_nw = 0;
    c->P.nw = (int)n;
    c->B.wall_vel = nullptr;
    c->B.wall_x0 = c->B.wall_v0 = nullptr;
    c->wall_vel_host.clear();
    c->P.variant &= ~kVariantMovingWall;
    if (n == 0) {
      c->B.wallP = nullptr;
      c->B.wall_id = nullptr;
      c->B.wall_xyz = nullptr;
      c->B.wallI = nullptr;
      CK(cudaMemsetAsync(c->B.wall_cb, 0, ((size_t)c->P.ncell + 1) * 4, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      return leave(c);
    }
    auto A = [&](size_t bytes) { return dev_alloc(c, bytes, c->wall_blocks); };
    const size_t ts = tsize(c);
    c->B.wallP = A(n * (d == 3 ? 4 : 2) * ts);
    c->B.wall_id = (uint32_t*)A(n * 4);
    c->B.wall_xyz = (double*)A(n * 3 * 8);
    c->B.wallI = c->precision == SPH_MIXED ? A(n * (d == 3 ? 16 : 8)) : nullptr;
    c->B.wall_vel = moving ? A(n * (d == 3 ? 4 : 2) * ts) : nullptr;
    std::vector<Block> tmp;
    DevBuffers W = c->B;
    // the walls as given, kept for translating walls: positions SoA (3 n),
    // then the velocities SoA (3 n) when moving
    W.io = (double*)A(n * (moving ? 6 : 3) * 8);
    for (int p = 0; p < 2; ++p) {
      W.keys[p] = (uint32_t*)dev_alloc(c, n * 4, tmp);
      W.vals[p] = (uint32_t*)dev_alloc(c, n * 4, tmp);
    }
    const size_t tiles = (n + kSortTile - 1) / kSortTile;
    W.tile_hist = (uint32_t*)dev_alloc(c, tiles * ((size_t)1 << kMaxRadixBits) * 4, tmp);
    bool ok = c->B.wallP && c->B.wall_id && c->B.wall_xyz && W.io && W.keys[0] && W.keys[1] &&
              (c->precision != SPH_MIXED || c->B.wallI) && (!moving || c->B.wall_vel) &&
              W.vals[0] && W.vals[1] && W.tile_hist;
    if (!ok) {
      dev_free_list(c, tmp);
      dev_free_list(c, c->wall_blocks);
      c->P.nw = 0;
      c->B.wall_vel = nullptr;
      return set_err(c, SPH_E_OOM, "device allocation failed (wall buffers)");
    }
    // host AoS -> wall_xyz (scratch here) -> SoA [x | y | z] staging
    CK(cudaMemcpyAsync(c->B.wall_xyz, pos, n * d * 8, cudaMemcpyHostToDevice, c->stream));
    double* soa[3] = {W.io, W.io + n, W.io + 2 * n};
    if (d == 2) CK(cudaMemsetAsync(W.io + 2 * n, 0, n * 8, c->stream));
    launch_deinterleave(c->B.wall_xyz, (int)n, d, soa, c->stream);
    if (moving) {
      // the AoS scratch is free again once the positions are deinterleaved
      CK(cudaMemcpyAsync(c->B.wall_xyz, vel, n * d * 8, cudaMemcpyHostToDevice, c->stream));
      double* vsoa[3] = {W.io + 3 * n, W.io + 4 * n, W.io + 5 * n};
      if (d == 2) CK(cudaMemsetAsync(W.io + 5 * n, 0, n * 8, c->stream));
      launch_deinterleave(c->B.wall_xyz, (int)n, d, vsoa, c->stream);
      c->P.variant |= kVariantMovingWall;
      c->wall_vel_host.assign(vel, vel + n * d);
    }
    c->B.wall_x0 = W.io;
    c->B.wall_v0 = moving ? W.io + 3 * n : nullptr;
    StageArgs a = args(c);
    a.B = W;
    if (c->precision == SPH_FP64)
      enqueue_wall_setup_fp64(a, c->stream);
    else
      enqueue_wall_setup_mixed(a, c->stream);
    CK(cudaGetLastError());
    CK(invalidate_lists(c));
    CK(cudaStreamSynchronize(c->stream));
    dev_free_list(c, tmp);
    c->cap_nw = n;
    return leave(c);
  }
  return set_err(c, SPH_E_INVALID, "unknown particle kind");
}

// ---------------------------------------------------------------------------
// Checkpoints: the schedule scalars and the live state in storage order
// (positions, velocities, densities, carried density rates, prior
// accelerations, user ids, binned cell keys), behind a header that names the
// setup it belongs to.
namespace {
constexpr char kCkptMagic[8] = {'S', 'P', 'H', 'C', 'K', 'P', 'T', '1'};
constexpr int32_t kCkptVersion = 4;

struct CkptHeader {
  char magic[8];
  int32_t version, dim, precision, variant;
  int64_t n, nw, ncell;
  int32_t nx, ny, nz, pad_;
  double h, cs, rho0, c0, mu, U_ref, m, V, wall_vmax, wall_omega;
  double lo[3], g[3];
  uint64_t scalars_bytes;
};

void ckpt_header(const sph_ctx* c, CkptHeader* hd) {
  memset(hd, 0, sizeof(*hd));
  memcpy(hd->magic, kCkptMagic, 8);
  const Params& P = c->P;
  hd->version = kCkptVersion;
  hd->dim = P.dim;
  hd->precision = c->precision;
  hd->variant = P.variant;
  hd->n = P.n;
  hd->nw = P.nw;
  hd->ncell = P.ncell;
  hd->nx = P.nx;
  hd->ny = P.ny;
  hd->nz = P.nz;
  hd->h = P.h;
  hd->cs = P.cs;
  hd->rho0 = P.rho0;
  hd->c0 = P.c0;
  hd->mu = P.mu;
  hd->U_ref = P.U_ref;
  hd->m = P.m;
  hd->V = P.V;
  hd->wall_vmax = P.wall_vmax;
  hd->wall_omega = P.wall_omega;
  for (int k = 0; k < 3; ++k) {
    hd->lo[k] = P.lo[k];
    hd->g[k] = P.g[k];
  }
  hd->scalars_bytes = sizeof(DevScalars);
}

// bytes per fluid particle: x, v (double), rho (double), drho (pair type),
// a_prior (pair type), position at the rebuild (record frame, pair type),
// drift budget (float), id, binned key
size_t ckpt_per_particle(const sph_ctx* c) {
  const size_t d = (size_t)c->P.dim, ts = tsize(c);
  return 2 * d * 8 + 8 + ts + d * ts + d * ts + 4 + 4 + 4;
}
}  // namespace

size_t sph_checkpoint_bytes(const sph_ctx* c) {
  if (!c || !c->fluid_set) return 0;
  return sizeof(CkptHeader) + sizeof(DevScalars) + (size_t)c->P.n * ckpt_per_particle(c);
}

int sph_checkpoint_save(sph_ctx* c, void* buf, size_t bytes) {
  TraceRange trace_("sph_checkpoint_save");
  if (!c) return SPH_E_INVALID;
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  if (!buf || bytes < sph_checkpoint_bytes(c))
    return set_err(c, SPH_E_INVALID, "checkpoint buffer missing or too small");
  int rc = enter(c);
  if (rc) return rc;
  DevScalars hs;
  rc = read_scalars(c, &hs);
  if (rc) return rc;
  CkptHeader hd;
  ckpt_header(c, &hd);
  char* p = (char*)buf;
  memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  memcpy(p, &hs, sizeof(hs));
  p += sizeof(hs);
  const size_t n = (size_t)c->P.n, ts = tsize(c);
  const int d = c->P.dim, par = hs.par;
  const DevBuffers& B = c->B;
  auto D2H = [&](const void* src, size_t nbytes) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(p, src, nbytes, cudaMemcpyDeviceToHost, c->stream);
    p += nbytes;
    return e;
  };
  for (int k = 0; k < d; ++k) CK(D2H(B.x[par][k], n * 8));
  for (int k = 0; k < d; ++k) CK(D2H(B.v[par][k], n * 8));
  CK(D2H(B.rho[par], n * 8));
  CK(D2H(B.drho[par], n * ts));
  for (int k = 0; k < d; ++k) CK(D2H(B.aprior[k], n * ts));
  for (int k = 0; k < d; ++k) CK(D2H(B.xreb[k], n * ts));
  CK(D2H(B.bud, n * 4));
  CK(D2H(B.id[par], n * 4));
  CK(D2H(B.keys[B.sorted_buf], n * 4));
  CK(cudaStreamSynchronize(c->stream));
  rc = leave(c);
  return rc ? rc : flags_status(c, hs);
}

int sph_checkpoint_load(sph_ctx* c, const void* buf, size_t bytes) {
  TraceRange trace_("sph_checkpoint_load");
  if (!c) return SPH_E_INVALID;
  if (!buf || bytes < sizeof(CkptHeader) + sizeof(DevScalars))
    return set_err(c, SPH_E_INVALID, "checkpoint buffer missing or too small");
  CkptHeader hd, mine;
  memcpy(&hd, buf, sizeof(hd));
  if (memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.version != kCkptVersion ||
      hd.scalars_bytes != sizeof(DevScalars))
    return set_err(c, SPH_E_INVALID, "not a checkpoint of this library version");
  ckpt_header(c, &mine);
  const bool same = hd.dim == mine.dim && hd.precision == mine.precision &&
                    hd.variant == mine.variant && hd.nw == mine.nw && hd.ncell == mine.ncell &&
                    hd.nx == mine.nx && hd.ny == mine.ny && hd.nz == mine.nz &&
                    hd.h == mine.h && hd.cs == mine.cs && hd.rho0 == mine.rho0 &&
                    hd.c0 == mine.c0 && hd.mu == mine.mu && hd.U_ref == mine.U_ref &&
                    hd.m == mine.m && hd.V == mine.V && hd.wall_vmax == mine.wall_vmax &&
                    hd.wall_omega == mine.wall_omega &&
                    memcmp(hd.lo, mine.lo, sizeof(hd.lo)) == 0 &&
                    memcmp(hd.g, mine.g, sizeof(hd.g)) == 0;
  if (!same)
    return set_err(c, SPH_E_INVALID,
                   "checkpoint of a different setup (domain, material, precision, walls, "
                   "translation or method options)");
  if (hd.n <= 0 || hd.n >= (1ll << 25)) return set_err(c, SPH_E_INVALID, "bad particle count");
  const size_t n = (size_t)hd.n;
  if (bytes < sizeof(CkptHeader) + sizeof(DevScalars) + n * ckpt_per_particle(c))
    return set_err(c, SPH_E_INVALID, "checkpoint buffer too small for its particle count");
  {
    // the ids and binned keys index device arrays: check them on the host
    // (keys in the grid and in storage order, ids a permutation)
    const char* q = (const char*)buf + sizeof(CkptHeader) + sizeof(DevScalars) +
                    n * (ckpt_per_particle(c) - 8);
    const uint32_t* ids = (const uint32_t*)q;
    const uint32_t* keys = (const uint32_t*)(q + n * 4);
    std::vector<uint8_t> seen(n, 0);
    for (size_t k = 0; k < n; ++k) {
      if (keys[k] >= c->P.ncell || (k > 0 && keys[k] < keys[k - 1]) || ids[k] >= n ||
          seen[ids[k]])
        return set_err(c, SPH_E_INVALID, "checkpoint with bad cell keys or particle ids");
      seen[ids[k]] = 1;
    }
  }
  int rc = enter(c);
  if (rc) return rc;
  rc = alloc_fluid(c, n);
  if (rc) return rc;
  drop_graph(c);
  c->P.n = (int)n;
  configure_launch(c);
  DevScalars hs;
  const char* p = (const char*)buf + sizeof(hd);
  memcpy(&hs, p, sizeof(hs));
  p += sizeof(hs);
  // the state goes to copy 0; the lists are built anew below
  hs.par = 0;
  const size_t ts = tsize(c);
  const int d = c->P.dim;
  DevBuffers& B = c->B;
  auto H2D = [&](void* dst, size_t nbytes) -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(dst, p, nbytes, cudaMemcpyHostToDevice, c->stream);
    p += nbytes;
    return e;
  };
  for (int k = 0; k < d; ++k) CK(H2D(B.x[0][k], n * 8));
  for (int k = 0; k < d; ++k) CK(H2D(B.v[0][k], n * 8));
  CK(H2D(B.rho[0], n * 8));
  CK(H2D(B.drho[0], n * ts));
  for (int k = 0; k < d; ++k) CK(H2D(B.aprior[k], n * ts));
  for (int k = 0; k < d; ++k) CK(H2D(B.xreb[k], n * ts));
  CK(H2D(B.bud, n * 4));
  CK(H2D(B.id[0], n * 4));
  CK(H2D(B.keys[B.sorted_buf], n * 4));
  for (int k = 0; k < d; ++k) CK(cudaMemsetAsync(B.acc[k], 0, n * ts, c->stream));
  CK(cudaMemsetAsync(B.sigma, 0, n * ts, c->stream));
  CK(cudaMemcpyAsync(B.sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, c->stream));
  launch_cell_offsets(B.keys[B.sorted_buf], (int)n, c->P.ncell, B.cell_begin, B.sc, 0, 0,
                      c->stream);
  if (c->precision == SPH_MIXED) enqueue_units_mixed(args(c), c->stream);
  // translating walls: binned at the saved rebuild time, moved to the saved time
  if ((c->P.variant & kVariantTranslatingWall) && c->P.nw > 0) {
    if (c->precision == SPH_FP64)
      enqueue_wall_rebin_fp64(args(c), c->stream, 1);
    else
      enqueue_wall_rebin_mixed(args(c), c->stream, 1);
  }
  // neighbour lists from the restored positions with the saved skin (a list
  // that overflowed before the save stays marked bad)
  if (!hs.list_bad) {
    if (c->precision == SPH_FP64)
      enqueue_restore_lists_fp64(args(c), c->stream);
    else
      enqueue_restore_lists_mixed(args(c), c->stream);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  c->fluid_set = true;
  return leave(c);
}

int sph_set_wall_motion(sph_ctx* c, const uint8_t* moves, double omega,
                        const double* amplitude) {
  TraceRange trace_("sph_set_wall_motion");
  if (!c) return SPH_E_INVALID;
  if (!std::isfinite(omega)) return set_err(c, SPH_E_INVALID, "omega is not finite");
  const size_t n = (size_t)c->P.nw;
  const int d = c->P.dim;
  if (amplitude)
    for (size_t q = 0; q < n * (size_t)d; ++q)
      if (!std::isfinite(amplitude[q]))
        return set_err(c, SPH_E_INVALID, "wall amplitude is not finite");
  int rc = enter(c);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  drop_graph(c);
  dev_free_list(c, c->trans_blocks);
  clear_translation(c);
  if (n == 0) return leave(c);
  bool any = false, osc = false;
  double vmax = 0.0;
  if (moves) {
    for (size_t u = 0; u < n; ++u) {
      if (!moves[u]) continue;
      any = true;
      double v2 = 0.0, a2 = 0.0;
      for (int k = 0; k < d; ++k) {
        if (!c->wall_vel_host.empty())
          v2 += c->wall_vel_host[u * d + k] * c->wall_vel_host[u * d + k];
        if (amplitude) a2 += amplitude[u * d + k] * amplitude[u * d + k];
      }
      if (a2 > 0.0 && omega != 0.0) osc = true;
      vmax = std::max(vmax, std::sqrt(v2) + std::sqrt(a2) * std::fabs(omega));
    }
  }
  // walls given no velocity and no oscillation are at rest: nothing moves
  if (!c->B.wall_v0 && !osc) any = false;
  auto A = [&](size_t bytes) { return dev_alloc(c, bytes, c->trans_blocks); };
  const size_t rec = n * (d == 3 ? 4 : 2) * tsize(c);
  uint8_t* dm = any ? (uint8_t*)A(n) : nullptr;
  c->B.wall_io = (double*)A(n * 3 * 8);
  c->B.wall_key = (uint32_t*)A(n * 4);
  for (int p = 0; p < 2; ++p) {
    c->B.wkeys[p] = (uint32_t*)A(n * 4);
    c->B.wvals[p] = (uint32_t*)A(n * 4);
  }
  const size_t tiles = (n + kSortTile - 1) / kSortTile;
  c->B.wtile_hist = (uint32_t*)A(tiles * ((size_t)1 << kMaxRadixBits) * 4);
  double* amp = osc ? (double*)A(n * 3 * 8) : nullptr;
  void* acc = osc ? A(rec) : nullptr;
  const bool need_vel = osc && !c->B.wall_vel;
  void* vel = need_vel ? A(rec) : nullptr;
  double* v0 = need_vel ? (double*)A(n * 3 * 8) : nullptr;
  const bool ok = (!any || dm) && c->B.wall_io && c->B.wall_key && c->B.wkeys[0] &&
                  c->B.wkeys[1] && c->B.wvals[0] && c->B.wvals[1] && c->B.wtile_hist &&
                  (!osc || (amp && acc)) && (!need_vel || (vel && v0));
  if (!ok) {
    dev_free_list(c, c->trans_blocks);
    clear_translation(c);
    return set_err(c, SPH_E_OOM, "device allocation failed (translating walls)");
  }
  if (any) {
    CK(cudaMemcpyAsync(dm, moves, n, cudaMemcpyHostToDevice, c->stream));
    c->B.wall_moves = dm;
    c->P.variant |= kVariantTranslatingWall;
    c->P.wall_vmax = vmax;
  }
  if (osc) {
    // amplitudes: host AoS -> wall_io (scratch here) -> SoA
    CK(cudaMemcpyAsync(c->B.wall_io, amplitude, n * d * 8, cudaMemcpyHostToDevice, c->stream));
    double* soa[3] = {amp, amp + n, amp + 2 * n};
    if (d == 2) CK(cudaMemsetAsync(amp + 2 * n, 0, n * 8, c->stream));
    launch_deinterleave(c->B.wall_io, (int)n, d, soa, c->stream);
    c->B.wall_amp = amp;
    c->B.wall_acc = acc;
    if (need_vel) {
      // walls given without velocities: zero base velocity, records owned here
      CK(cudaMemsetAsync(v0, 0, n * 3 * 8, c->stream));
      c->B.wall_vel = vel;
      c->B.wall_v0 = v0;
      c->P.variant |= kVariantMovingWall;
      c->motion_owns_vel = true;
    }
    c->P.variant |= kVariantAccelWall;
    c->P.wall_omega = omega;
  }
  // walls binned again where they are now (back at their given positions
  // when none translates)
  if (c->precision == SPH_FP64)
    enqueue_wall_rebin_fp64(args(c), c->stream, 0);
  else
    enqueue_wall_rebin_mixed(args(c), c->stream, 0);
  CK(cudaGetLastError());
  CK(invalidate_lists(c));
  CK(cudaStreamSynchronize(c->stream));
  return leave(c);
}

int sph_set_wall_translation(sph_ctx* c, const uint8_t* moves) {
  return sph_set_wall_motion(c, moves, 0.0, nullptr);
}

int sph_step(sph_ctx* c, int n) {
  TraceRange trace_("sph_step");
  if (!c) return SPH_E_INVALID;
  if (n < 0) return set_err(c, SPH_E_INVALID, "negative step count");
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  if (n == 0) return SPH_OK;
  int rc = enter(c);
  if (rc) return rc;
  if (c->use_graph) {
    if (!c->graph_exec) {
      cudaError_t e = capture_step_graph(c, &c->graph);
      if (e != cudaSuccess) {
        c->graph = nullptr;
        return cuda_err(c, e, "graph capture");
      }
      e = cudaGraphInstantiate(&c->graph_exec, c->graph, 0);
      if (e != cudaSuccess) {
        drop_graph(c);
        return cuda_err(c, e, "graph instantiate");
      }
    }
    for (int i = 0; i < n; ++i) CK(cudaGraphLaunch(c->graph_exec, c->stream));
  } else {
    for (int i = 0; i < n; ++i) enqueue_step(c, c->stream);
    CK(cudaGetLastError());
  }
  return leave(c);
}

int sph_synchronize(sph_ctx* c, double timeout_s) {
  if (!c) return SPH_E_INVALID;
  CK(cudaEventRecord(c->ev_out, c->stream));
  if (timeout_s > 0) {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      cudaError_t e = cudaEventQuery(c->ev_out);
      if (e == cudaSuccess) break;
      if (e != cudaErrorNotReady) return cuda_err(c, e, "sph_synchronize");
      double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > timeout_s) return set_err(c, SPH_E_TIMEOUT, "queued work did not finish in time");
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  }
  return sync_status(c);
}

int sph_get_fields(sph_ctx* c, unsigned mask, double* out) {
  TraceRange trace_("sph_get_fields");
  if (!c || (!out && mask)) return SPH_E_INVALID;
  if (mask & ~0xffu) return set_err(c, SPH_E_INVALID, "unknown field bit");
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  int rc = enter(c);
  if (rc) return rc;
  DevScalars hs;
  rc = read_scalars(c, &hs);
  if (rc) return rc;
  const int par = hs.par, d = c->P.dim, n = c->P.n;
  const DevBuffers& B = c->B;
  const int isf = c->precision == SPH_MIXED;
  double* o = out;
  for (unsigned bit = 1; bit <= SPH_F_SIGMA; bit <<= 1) {
    if (!(mask & bit)) continue;
    int comps = 1;
    switch (bit) {
      case SPH_F_POS:
        comps = d;
        rc = scatter_out(c, B.x[par][0], B.x[par][1], B.x[par][2], 0, 1, 0, d, par, o);
        break;
      case SPH_F_VEL:
        comps = d;
        rc = scatter_out(c, B.v[par][0], B.v[par][1], B.v[par][2], 0, 1, 0, d, par, o);
        break;
      case SPH_F_RHO:
        rc = scatter_out(c, B.rho[par], nullptr, nullptr, 0, 1, 0, 1, par, o);
        break;
      case SPH_F_P:
        // pressure of the last first half-step, kept in the records of buffer 0
        if (d == 3)
          rc = scatter_out(c, B.rec[0], nullptr, nullptr, isf, 8, 3, 1, par, o);
        else
          rc = scatter_out(c, B.rec_s[0], nullptr, nullptr, isf, 2, 0, 1, par, o);
        break;
      case SPH_F_DRHO:
        rc = scatter_out(c, B.drho[par], nullptr, nullptr, isf, 1, 0, 1, par, o);
        break;
      case SPH_F_ACC:
        comps = d;
        rc = scatter_out(c, B.acc[0], B.acc[1], B.acc[2], isf, 1, 0, d, par, o);
        break;
      case SPH_F_APRIOR:
        comps = d;
        rc = scatter_out(c, B.aprior[0], B.aprior[1], B.aprior[2], isf, 1, 0, d, par, o);
        break;
      case SPH_F_SIGMA:
        rc = scatter_out(c, B.sigma, nullptr, nullptr, isf, 1, 0, 1, par, o);
        break;
    }
    if (rc) return rc;
    o += (size_t)n * comps;
  }
  rc = leave(c);
  if (rc) return rc;
  return flags_status(c, hs);
}

int sph_get_scalars(sph_ctx* c, double* t, double* dt_ad, double* dt_ac, long* n_ac,
                    long* n_adv) {
  if (!c) return SPH_E_INVALID;
  int rc = enter(c);
  if (rc) return rc;
  DevScalars hs;
  rc = read_scalars(c, &hs);
  if (rc) return rc;
  if (t) *t = hs.t;
  if (dt_ad) *dt_ad = hs.dt_ad;
  if (dt_ac) *dt_ac = hs.dt_ac;
  if (n_ac) *n_ac = (long)hs.n_ac;
  if (n_adv) *n_adv = (long)hs.n_adv;
  return flags_status(c, hs);
}

size_t sph_count(const sph_ctx* c, int kind) {
  if (!c) return 0;
  return kind == SPH_WALL ? (size_t)c->P.nw : (size_t)c->P.n;
}

size_t sph_cell_count(const sph_ctx* c) { return c ? (size_t)c->P.ncell : 0; }

int sph_debug_neighbour_state(sph_ctx* c, uint32_t* keys, uint32_t* perm, uint32_t* ids,
                              uint32_t* cell_begin) {
  if (!c) return SPH_E_INVALID;
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  int rc = enter(c);
  if (rc) return rc;
  DevScalars hs;
  rc = read_scalars(c, &hs);
  if (rc) return rc;
  const size_t n = c->P.n;
  const int sb = c->B.sorted_buf;
  if (keys) CK(cudaMemcpyAsync(keys, c->B.keys[sb], n * 4, cudaMemcpyDeviceToHost, c->stream));
  if (perm) CK(cudaMemcpyAsync(perm, c->B.vals[sb], n * 4, cudaMemcpyDeviceToHost, c->stream));
  if (ids) CK(cudaMemcpyAsync(ids, c->B.id[hs.par], n * 4, cudaMemcpyDeviceToHost, c->stream));
  if (cell_begin)
    CK(cudaMemcpyAsync(cell_begin, c->B.cell_begin, ((size_t)c->P.ncell + 1) * 4,
                       cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  rc = leave(c);
  if (rc) return rc;
  return flags_status(c, hs);
}

int sph_debug_neighbour_stats(sph_ctx* c, uint32_t* cnt_fluid, uint32_t* cnt_wall,
                              uint64_t* hash) {
  if (!c || !cnt_fluid || !cnt_wall || !hash) return SPH_E_INVALID;
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  int rc = enter(c);
  if (rc) return rc;
  const size_t n = c->P.n;
  std::vector<Block> tmp;
  uint32_t* cf = (uint32_t*)dev_alloc(c, n * 4, tmp);
  uint32_t* cw = (uint32_t*)dev_alloc(c, n * 4, tmp);
  unsigned long long* hs = (unsigned long long*)dev_alloc(c, n * 8, tmp);
  if (!cf || !cw || !hs) {
    dev_free_list(c, tmp);
    return set_err(c, SPH_E_OOM, "device allocation failed (neighbour stats)");
  }
  launch_neighbour_stats(c->P, c->L, c->B, c->B.wall_xyz, cf, cw, hs, c->stream);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt_fluid, cf, n * 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt_wall, cw, n * 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hash, hs, n * 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dev_free_list(c, tmp);
  if (e != cudaSuccess) return cuda_err(c, e, "sph_debug_neighbour_stats");
  rc = leave(c);
  if (rc) return rc;
  return sync_status(c);
}

// ---------------------------------------------------------------------------
// State by user-id range and the schedule scalars: what a decomposition of one
// tank into slabs exchanges between the contexts of its ranks.
namespace {
int state_range(sph_ctx* c, uint32_t id0, size_t m, double* const host[5], int put) {
  if (!c) return SPH_E_INVALID;
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  if ((size_t)id0 + m > (size_t)c->P.n) return set_err(c, SPH_E_INVALID, "id range beyond n");
  if (m == 0) return SPH_OK;
  int rc = enter(c);
  if (rc) return rc;
  const int d = c->P.dim;
  const int is_float = c->precision == SPH_MIXED ? 1 : 0;
  for (int f = 0; f < 5; ++f) {
    if (!host[f]) continue;
    const size_t bytes = m * (size_t)(f == 0 || f == 1 || f == 4 ? d : 1) * 8;
    if (put) {
      CK(cudaMemcpyAsync(c->B.io, host[f], bytes, cudaMemcpyHostToDevice, c->stream));
      launch_state_range(c->P, c->L, c->B, id0, (uint32_t)m, c->B.io, f, 1, is_float, c->stream);
    } else {
      launch_state_range(c->P, c->L, c->B, id0, (uint32_t)m, c->B.io, f, 0, is_float, c->stream);
      CK(cudaMemcpyAsync(host[f], c->B.io, bytes, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaGetLastError());
    // the staging buffer is reused by the next field
    CK(cudaStreamSynchronize(c->stream));
  }
  rc = leave(c);
  if (rc) return rc;
  return sync_status(c);
}
}  // namespace

int sph_get_state_range(sph_ctx* c, uint32_t id0, size_t m, double* pos, double* vel,
                        double* rho, double* drho, double* aprior) {
  TraceRange tr("sph_get_state_range");
  double* const h[5] = {pos, vel, rho, drho, aprior};
  return state_range(c, id0, m, h, 0);
}

int sph_put_state_range(sph_ctx* c, uint32_t id0, size_t m, const double* pos, const double* vel,
                        const double* rho, const double* drho, const double* aprior) {
  TraceRange tr("sph_put_state_range");
  double* const h[5] = {(double*)pos, (double*)vel, (double*)rho, (double*)drho,
                        (double*)aprior};
  return state_range(c, id0, m, h, 1);
}

namespace {
int state_rows_device(sph_ctx* c, uint32_t id0, size_t m, double* rows, int put) {
  if (!c || (m > 0 && !rows)) return SPH_E_INVALID;
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  if ((size_t)id0 + m > (size_t)c->P.n) return set_err(c, SPH_E_INVALID, "id range beyond n");
  if (m == 0) return SPH_OK;
  int rc = enter(c);
  if (rc) return rc;
  launch_state_rows(c->P, c->L, c->B, id0, (uint32_t)m, rows, put,
                    c->precision == SPH_MIXED ? 1 : 0, c->stream);
  CK(cudaGetLastError());
  return leave(c);
}
}  // namespace

int sph_get_state_rows_device(sph_ctx* c, uint32_t id0, size_t m, double* rows) {
  return state_rows_device(c, id0, m, rows, 0);
}

int sph_put_state_rows_device(sph_ctx* c, uint32_t id0, size_t m, const double* rows) {
  return state_rows_device(c, id0, m, (double*)rows, 1);
}

int sph_owned_vmax2_device(sph_ctx* c, uint32_t n_own, double* vmax2) {
  if (!c || !vmax2) return SPH_E_INVALID;
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  int rc = enter(c);
  if (rc) return rc;
  CK(cudaMemsetAsync(vmax2, 0, sizeof(double), c->stream));
  launch_vmax_owned(c->P, c->L, c->B, n_own, (unsigned long long*)vmax2, c->stream);
  CK(cudaGetLastError());
  return leave(c);
}

int sph_set_vmax2_device(sph_ctx* c, const double* vmax2) {
  if (!c || !vmax2) return SPH_E_INVALID;
  int rc = enter(c);
  if (rc) return rc;
  CK(cudaMemcpyAsync((char*)c->B.sc + offsetof(DevScalars, vmax2_cur), vmax2, sizeof(double),
                     cudaMemcpyDeviceToDevice, c->stream));
  return leave(c);
}

int sph_get_schedule(sph_ctx* c, double sched[8]) {
  if (!c || !sched) return SPH_E_INVALID;
  int rc = enter(c);
  if (rc) return rc;
  DevScalars hs;
  rc = read_scalars(c, &hs);
  if (rc) return rc;
  sched[0] = hs.t;
  sched[1] = hs.tau;
  sched[2] = hs.dt_ad;
  sched[3] = hs.dt_ac;
  sched[4] = (double)hs.n_ac;
  sched[5] = (double)hs.n_adv;
  sched[6] = (double)hs.started;
  sched[7] = __longlong_as_double_host((long long)hs.vmax2_cur);
  return flags_status(c, hs);
}

int sph_set_schedule(sph_ctx* c, const double sched[8]) {
  if (!c || !sched) return SPH_E_INVALID;
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  for (int k = 0; k < 8; ++k)
    if (!std::isfinite(sched[k])) return set_err(c, SPH_E_INVALID, "schedule value not finite");
  if (!(sched[7] >= 0) || !(sched[1] >= 0) || !(sched[2] >= 0) || !(sched[3] >= 0))
    return set_err(c, SPH_E_INVALID, "negative schedule value");
  // only where the next step begins an advection step (its rebuild sets the
  // neighbour structure, lists and budgets anew)
  if (sched[6] != 0.0 && !(sched[1] >= sched[2]))
    return set_err(c, SPH_E_INVALID, "schedule must be at an advection-step boundary (tau >= dt_ad)");
  int rc = enter(c);
  if (rc) return rc;
  DevScalars hs;
  rc = read_scalars(c, &hs);
  if (rc) return rc;
  hs.t = sched[0];
  hs.tau = sched[1];
  hs.dt_ad = sched[2];
  hs.dt_ac = sched[3];
  hs.n_ac = (long long)sched[4];
  hs.n_adv = (long long)sched[5];
  hs.started = sched[6] != 0.0 ? 1 : 0;
  hs.vmax2_cur = (unsigned long long)__double_as_longlong_host(sched[7]);
  CK(cudaMemcpyAsync(c->B.sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return leave(c);
}

int sph_set_vmax2(sph_ctx* c, double vmax2) {
  if (!c) return SPH_E_INVALID;
  if (!(vmax2 >= 0) || !std::isfinite(vmax2))
    return set_err(c, SPH_E_INVALID, "vmax2 must be finite and non-negative");
  int rc = enter(c);
  if (rc) return rc;
  const unsigned long long bits = (unsigned long long)__double_as_longlong_host(vmax2);
  CK(cudaMemcpyAsync((char*)c->B.sc + offsetof(DevScalars, vmax2_cur), &bits, sizeof(bits),
                     cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return leave(c);
}

int sph_owned_vmax2(sph_ctx* c, uint32_t n_own, double* vmax2) {
  if (!c || !vmax2) return SPH_E_INVALID;
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  int rc = enter(c);
  if (rc) return rc;
  unsigned long long* out = c->B.u64_io;
  CK(cudaMemsetAsync(out, 0, sizeof(*out), c->stream));
  launch_vmax_owned(c->P, c->L, c->B, n_own, out, c->stream);
  CK(cudaGetLastError());
  unsigned long long bits = 0;
  CK(cudaMemcpyAsync(&bits, out, sizeof(bits), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *vmax2 = __longlong_as_double_host((long long)bits);
  rc = leave(c);
  if (rc) return rc;
  return sync_status(c);
}

int sph_debug_list_lengths(sph_ctx* c, uint32_t* lengths) {
  if (!c || !lengths) return SPH_E_INVALID;
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  int rc = enter(c);
  if (rc) return rc;
  const size_t n = c->P.n;
  if (c->P.use_list)
    CK(cudaMemcpyAsync(lengths, c->B.nl_cnt, n * 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (!c->P.use_list) memset(lengths, 0, n * 4);
  // a count word packs the fluid run (bits 0..15) and the wall run (16..31)
  for (size_t k = 0; k < n && c->P.use_list; ++k)
    lengths[k] = (lengths[k] & 0xFFFFu) + (lengths[k] >> 16);
  rc = leave(c);
  if (rc) return rc;
  return sync_status(c);
}

int sph_profile_stages(sph_ctx* c, int n, double* ms, long* rebuilds) {
  TraceRange trace_("sph_profile_stages");
  if (!c || !ms || n < 0) return SPH_E_INVALID;
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  int rc = enter(c);
  if (rc) return rc;
  DevScalars before, after;
  rc = read_scalars(c, &before);
  if (rc) return rc;
  cudaEvent_t ev[kStages + 1];
  for (int k = 0; k <= kStages; ++k) CK(cudaEventCreate(&ev[k]));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    if (c->precision == SPH_FP64)
      enqueue_step_fp64(args(c), c->stream, ev);
    else
      enqueue_step_mixed(args(c), c->stream, ev);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[kStages]);
    for (int k = 0; k < kStages && e == cudaSuccess; ++k) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      ms[k] += t;
    }
  }
  for (int k = 0; k <= kStages; ++k) cudaEventDestroy(ev[k]);
  if (e != cudaSuccess) return cuda_err(c, e, "sph_profile_stages");
  rc = read_scalars(c, &after);
  if (rc) return rc;
  if (rebuilds) *rebuilds = (long)(after.n_adv - before.n_adv);
  rc = leave(c);
  if (rc) return rc;
  return flags_status(c, after);
}

long sph_kernels_per_step(const sph_ctx* cc) {
  if (!cc) return -1;
  sph_ctx* c = const_cast<sph_ctx*>(cc);
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return -1;
  enqueue_step(c, c->stream);
  if (cudaStreamEndCapture(c->stream, &g) != cudaSuccess || !g) return -1;
  size_t count = 0;
  long kernels = -1;
  if (cudaGraphGetNodes(g, nullptr, &count) == cudaSuccess) {
    std::vector<cudaGraphNode_t> nodes(count);
    if (cudaGraphGetNodes(g, nodes.data(), &count) == cudaSuccess) {
      kernels = 0;
      for (auto nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
      }
    }
  }
  cudaGraphDestroy(g);
  return kernels;
}

int sph_set_option(sph_ctx* c, int option, long value) {
  if (!c) return SPH_E_INVALID;
  const int old_sorted = c->B.sorted_buf;
  const int old_list = c->P.use_list;
  switch (option) {
    case SPH_OPT_RECORD_DIAGNOSTICS:
      c->P.diag = value ? 1 : 0;
      break;
    case SPH_OPT_USE_GRAPH:
      c->use_graph = value != 0;
      break;
    case SPH_OPT_BLOCK:
      if (value < 64 || value > 256 || value % 32)
        return set_err(c, SPH_E_INVALID, "block size must be 64..256, a multiple of 32");
      c->L.block_loop = (int)value;
      configure_launch(c);
      break;
    case SPH_OPT_NEIGHBOUR_LIST:
      c->P.use_list = value ? 1 : 0;
      break;
    case SPH_OPT_RADIX_BITS:
      if (value < 4 || value > kMaxRadixBits)
        return set_err(c, SPH_E_INVALID, "radix bits must be 4..11");
      c->L.radix_bits = (int)value;
      configure_launch(c);
      break;
    case SPH_OPT_DENSITY_RIEMANN:
      c->P.variant = value ? (c->P.variant & ~kVariantNoRiemann) : (c->P.variant | kVariantNoRiemann);
      break;
    case SPH_OPT_REINIT_BLENDED:
      c->P.variant = value ? (c->P.variant | kVariantBlended) : (c->P.variant & ~kVariantBlended);
      break;
    case SPH_OPT_TRANSPORT_CORRECTION:
      c->P.variant =
          value ? (c->P.variant | kVariantTransport) : (c->P.variant & ~kVariantTransport);
      break;
    default:
      return set_err(c, SPH_E_INVALID, "unknown option");
  }
  drop_graph(c);
  if (c->fluid_set && (c->B.sorted_buf != old_sorted || (c->P.use_list && !old_list))) {
    int rc = enter(c);
    if (rc) return rc;
    if (c->B.sorted_buf != old_sorted) {
      // the binned keys (and the last permutation) move to the buffer the
      // new pass count ends in
      const size_t n = (size_t)c->P.n;
      CK(cudaMemcpyAsync(c->B.keys[c->B.sorted_buf], c->B.keys[old_sorted], n * 4,
                         cudaMemcpyDeviceToDevice, c->stream));
      CK(cudaMemcpyAsync(c->B.vals[c->B.sorted_buf], c->B.vals[old_sorted], n * 4,
                         cudaMemcpyDeviceToDevice, c->stream));
    }
    if (c->P.use_list && !old_list) {
      // no list was built at the last rebuild: direct search until the next one
      const int one = 1;
      CK(cudaMemcpyAsync(&c->B.sc->list_bad, &one, sizeof(int), cudaMemcpyHostToDevice,
                         c->stream));
      CK(cudaStreamSynchronize(c->stream));
    }
    return leave(c);
  }
  return SPH_OK;
}

int sph_autotune(sph_ctx* c, int steps_per_trial, sph_tuning* best) {
  TraceRange trace_("sph_autotune");
  if (!c || !best || steps_per_trial < 1) return SPH_E_INVALID;
  if (!c->fluid_set) return set_err(c, SPH_E_STATE, "no fluid particles set");
  int rc = enter(c);
  if (rc) return rc;
  CK(cudaStreamSynchronize(c->stream));
  DevMem mem;
  mem.alloc = c->alloc;
  mem.has_alloc = c->has_alloc;
  mem.stream = c->stream;
  Snapshot snap;
  if (!snap.take(mem, {&c->fluid_blocks, &c->wall_blocks, &c->fixed_blocks, &c->trans_blocks}))
    return set_err(c, SPH_E_OOM, "device allocation failed (autotuner snapshot)");
  const LaunchCfg L0 = c->L;
  const Params P0 = c->P;
  const int sorted0 = c->B.sorted_buf;
  const bool graph0 = c->use_graph;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // back to the state and configuration of the call
  auto reset = [&]() -> int {
    drop_graph(c);
    if (snap.restore(c->stream) != cudaSuccess || cudaStreamSynchronize(c->stream) != cudaSuccess)
      return SPH_E_CUDA;
    c->L = L0;
    c->P = P0;
    c->B.sorted_buf = sorted0;
    c->use_graph = true;
    return SPH_OK;
  };
  auto apply = [&](const sph_tuning& t) -> int {
    int r = sph_set_option(c, SPH_OPT_BLOCK, t.block);
    if (!r) r = sph_set_option(c, SPH_OPT_RADIX_BITS, t.radix_bits);
    if (!r) r = sph_set_option(c, SPH_OPT_NEIGHBOUR_LIST, t.neighbour_list);
    return r;
  };
  auto trial = [&](const sph_tuning& t) -> double {
    double bestms = -1.0;
    for (int rep = 0; rep < 2; ++rep) {
      if (reset() || apply(t)) return -1.0;
      if (cudaEventRecord(e0, c->user_stream) != cudaSuccess) return -1.0;
      if (sph_step(c, steps_per_trial)) return -1.0;
      if (cudaEventRecord(e1, c->user_stream) != cudaSuccess) return -1.0;
      if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0;
      const double per = ms / steps_per_trial;
      if (bestms < 0 || per < bestms) bestms = per;
    }
    return bestms;
  };
  sph_tuning start{L0.block_loop, L0.radix_bits, P0.use_list, 0, 0.0};
  sph_tuning found = start;
  int search = e == cudaSuccess ? tune_search(start, trial, &found) : -1;
  // leave the context as it was, with the chosen configuration
  rc = reset();
  if (!rc) rc = apply(search == 0 ? found : start);
  c->use_graph = graph0;
  snap.drop(mem);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (search != 0)
    return rc ? rc : set_err(c, SPH_E_CUDA, "autotuner trial failed: " + c->err);
  if (rc) return rc;
  *best = found;
  return leave(c);
}

const char* sph_last_error(const sph_ctx* c) { return c ? c->err.c_str() : "null context"; }

void sph_destroy(sph_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  dev_free_list(c, c->fluid_blocks);
  dev_free_list(c, c->trans_blocks);
  dev_free_list(c, c->wall_blocks);
  dev_free_list(c, c->fixed_blocks);
  if (c->ev_in) cudaEventDestroy(c->ev_in);
  if (c->ev_out) cudaEventDestroy(c->ev_out);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // extern "C"
