// C ABI of batches of independent tanks (sph_create_batch, sph_batch_*):
// per-tank parameters, constants and schedules on the device, the shared
// particle / cell arrays with one range per tank, the static work lists, and
// CUDA-graph replay of the batched acoustic step.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <cstddef>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "sph.h"
#include "sph_host.cuh"
#include "sph_internal.cuh"
#include "sph_stages.cuh"

using namespace sphgb;

struct sph_batch {
  int T = 0;
  int dim = 2;
  int precision = SPH_MIXED;
  std::vector<Params> P;  // host copies of the per-tank parameters
  std::vector<double> dp;
  LaunchCfg L{};
  DevBuffers B{};
  BatchArgs A{};
  DevMem mem;
  cudaStream_t user_stream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  bool use_graph = true;
  size_t N = 0, NW = 0;
  uint32_t total_cells = 0;  // sum of (ncell + 1)
  std::vector<Block> fixed_blocks, fluid_blocks, wall_blocks;
  std::string err;
  bool fluid_set = false;
};

namespace {

// The neighbour lists name walls by their sorted slot: walls sorted anew
// outside a rebuild send every tank's loops to direct search until its next
// rebuild.
__global__ void kb_lists_bad(DevScalars* tsc, int T) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < T) tsc[t].list_bad = 1;
}

int set_err(sph_batch* b, int code, const std::string& msg) {
  if (b) b->err = msg;
  return code;
}

int cuda_err(sph_batch* b, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return SPH_OK;
  return set_err(b, SPH_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CKB(call)                                         \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_err(b, e_, #call); \
  } while (0)

size_t tsize(const sph_batch* b) { return b->precision == SPH_FP64 ? 8 : 4; }

void drop_graph(sph_batch* b) {
  if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->graph_exec = nullptr;
  b->graph = nullptr;
}

int enter(sph_batch* b) {
  CKB(cudaEventRecord(b->ev_in, b->user_stream));
  CKB(cudaStreamWaitEvent(b->mem.stream, b->ev_in, 0));
  return SPH_OK;
}
int leave(sph_batch* b) {
  CKB(cudaEventRecord(b->ev_out, b->mem.stream));
  CKB(cudaStreamWaitEvent(b->user_stream, b->ev_out, 0));
  return SPH_OK;
}

void configure_launch(sph_batch* b) {
  LaunchCfg& L = b->L;
  if (L.block_loop <= 0) L.block_loop = 128;
  L.blocks_loop = L.sms * (2048 / L.block_loop);
  L.block_stream = 256;
  L.blocks_stream = L.sms * 8;
  L.key_bits = bits_for(b->total_cells);
  L.radix_passes = radix_passes_for(L.key_bits, L.radix_bits);
  b->B.sorted_buf = L.radix_passes % 2;
}

BatchStageArgs args(const sph_batch* b) {
  BatchStageArgs a;
  a.A = b->A;
  a.B = b->B;
  a.B.binned = b->A.bkey;
  a.L = b->L;
  a.dim = b->dim;
  a.variants = 0;
  for (const auto& p : b->P) a.variants |= p.variant;
  return a;
}

void enqueue_step(sph_batch* b, cudaStream_t s, cudaEvent_t* ev = nullptr) {
  if (b->precision == SPH_FP64)
    enqueue_batch_step_fp64(args(b), s, ev);
  else
    enqueue_batch_step_mixed(args(b), s, ev);
}

// A static work list over every tank: tiles of `tile` slots of the fluid
// (walls = 0) or wall (walls = 1) ranges, offset chunks of every grid, and
// compacted bases equal to the ranges' first slots.
WorkList make_list(const sph_batch* b, int walls, int tile) {
  WorkList w;
  memset(&w, 0, sizeof(w));
  int tiles = 0, chunks = 0;
  for (int t = 0; t < b->T; ++t) {
    const Params& P = b->P[t];
    const int n = walls ? P.nw : P.n;
    w.tank[t] = t;
    w.tile_prefix[t] = tiles;
    w.chunk_prefix[t] = chunks;
    w.cbase[t] = walls ? P.woff : P.foff;
    tiles += (n + tile - 1) / tile;
    chunks += (int)((P.ncell + kOffsetsChunk - 1) / kOffsetsChunk);
  }
  w.count = b->T;
  w.tiles = tiles;
  w.chunks = chunks;
  w.m = walls ? (int)b->NW : (int)b->N;
  w.tile = tile;
  w.tile_prefix[b->T] = tiles;
  w.chunk_prefix[b->T] = chunks;
  return w;
}

// Uploads the per-tank parameters and the static lists, and refreshes the
// host-side sizes of the device view.
int upload_tables(sph_batch* b) {
  cudaStream_t s = b->mem.stream;
  CKB(cudaMemcpyAsync((void*)b->A.tP, b->P.data(), sizeof(Params) * b->T, cudaMemcpyHostToDevice,
                      s));
  const WorkList all = make_list(b, 0, b->L.block_loop);
  const WorkList wall = make_list(b, 1, 256);
  CKB(cudaMemcpyAsync(b->A.wl_all, &all, sizeof(WorkList), cudaMemcpyHostToDevice, s));
  CKB(cudaMemcpyAsync(b->A.wl_wall, &wall, sizeof(WorkList), cudaMemcpyHostToDevice, s));
  CKB(cudaStreamSynchronize(s));  // the host lists are stack temporaries
  b->A.tiles_max = all.tiles;
  b->A.chunks_max = all.chunks;
  b->A.n_total = (int)b->N;
  b->A.nw_total = (int)b->NW;
  return SPH_OK;
}

template <class T>
int upload_constants(sph_batch* b) {
  std::vector<stages::KC<T>> k(b->T);
  for (int t = 0; t < b->T; ++t) k[t] = stages::make_kc<T>(b->P[t]);
  CKB(cudaMemcpyAsync((void*)b->A.tK, k.data(), sizeof(stages::KC<T>) * b->T,
                      cudaMemcpyHostToDevice, b->mem.stream));
  CKB(cudaStreamSynchronize(b->mem.stream));
  return SPH_OK;
}

int read_scalars(sph_batch* b, std::vector<DevScalars>& hs) {
  hs.resize(b->T);
  CKB(cudaMemcpyAsync(hs.data(), b->A.tsc, sizeof(DevScalars) * b->T, cudaMemcpyDeviceToHost,
                      b->mem.stream));
  CKB(cudaStreamSynchronize(b->mem.stream));
  return SPH_OK;
}

int flags_status(sph_batch* b, const std::vector<DevScalars>& hs) {
  for (int t = 0; t < (int)hs.size(); ++t) {
    if (hs[t].flags & kFlagIndex)
      return set_err(b, SPH_E_INDEX, "an index check of the debug build failed (recorded on "
                                     "tank " + std::to_string(t) + ")");
    if (hs[t].flags & kFlagNonFinite)
      return set_err(b, SPH_E_NONFINITE,
                     "tank " + std::to_string(t) + ": a velocity or density became non-finite");
    if (hs[t].flags & kFlagOutOfDomain)
      return set_err(b, SPH_E_OUT_OF_DOMAIN,
                     "tank " + std::to_string(t) + ": a particle left the domain");
  }
  return SPH_OK;
}

int sync_status(sph_batch* b) {
  std::vector<DevScalars> hs;
  int rc = read_scalars(b, hs);
  if (rc) return rc;
  CKB(cudaGetLastError());
  return flags_status(b, hs);
}

int alloc_fluid(sph_batch* b, size_t n) {
  CKB(cudaStreamSynchronize(b->mem.stream));
  drop_graph(b);
  b->mem.release(b->fluid_blocks);
  DevBuffers& B = b->B;
  const size_t ts = tsize(b);
  const int d = b->dim;
  const size_t nn = n ? n : 1;
  auto Al = [&](size_t bytes) { return b->mem.get(bytes, b->fluid_blocks); };
  bool ok = true;
  for (int p = 0; p < 2; ++p) {
    for (int k = 0; k < 3; ++k) {
      B.x[p][k] = k < d ? (double*)Al(nn * 8) : nullptr;
      B.v[p][k] = k < d ? (double*)Al(nn * 8) : nullptr;
      ok &= k >= d || (B.x[p][k] && B.v[p][k]);
    }
    B.rho[p] = (double*)Al(nn * 8);
    B.drho[p] = Al(nn * ts);
    B.id[p] = (uint32_t*)Al(nn * 4);
    ok &= B.rho[p] && B.drho[p] && B.id[p];
  }
  for (int k = 0; k < 3; ++k) {
    B.aprior[k] = k < d ? Al(nn * ts) : nullptr;
    B.acc[k] = k < d ? Al(nn * ts) : nullptr;
    ok &= k >= d || (B.aprior[k] && B.acc[k]);
  }
  B.sigma = Al(nn * ts);
  B.sigma64 = (double*)Al(nn * 8);
  for (int k = 0; k < 3; ++k) {
    B.xreb[k] = k < d ? Al(nn * ts) : nullptr;
    ok &= k >= d || B.xreb[k];
  }
  B.bud = (float*)Al(nn * 4);
  B.brec = Al(nn * 4 * ts);
  ok &= B.sigma64 != nullptr && B.bud != nullptr && B.brec != nullptr;
  for (int p = 0; p < 2; ++p) {
    B.rec[p] = Al(nn * (d == 3 ? 8 : 4) * ts);
    B.rec_s[p] = d == 3 ? nullptr : Al(nn * 2 * ts);
    B.keys[p] = (uint32_t*)Al(nn * 4);
    B.vals[p] = (uint32_t*)Al(nn * 4);
    ok &= B.rec[p] && (d == 3 || B.rec_s[p]) && B.keys[p] && B.vals[p];
  }
  B.recI = b->precision == SPH_MIXED ? Al(nn * (d == 3 ? 16 : 8)) : nullptr;
  ok &= b->precision != SPH_MIXED || B.recI;
  const size_t warps = (nn + 31) / 32 + (size_t)b->T;  // per-warp list rows
  // two extra rows of 32 entries: the list walk prefetches two entries ahead
  B.nl = (uint32_t*)Al((warps * (size_t)b->P[0].list_cap + 2) * 32 * 4);
  B.nl_cnt = (uint32_t*)Al(nn * 4);
  b->A.bkey = (uint32_t*)Al(nn * 4);
  ok &= B.nl && B.nl_cnt && b->A.bkey;
  const size_t tiles = (nn + kSortTile - 1) / kSortTile;
  B.tile_hist = (uint32_t*)Al(tiles * ((size_t)1 << kMaxRadixBits) * 4);
  B.io = (double*)Al(nn * 3 * 8);
  ok &= B.sigma && B.tile_hist && B.io;
  if (!ok) {
    b->mem.release(b->fluid_blocks);
    return set_err(b, SPH_E_OOM, "device allocation failed (fluid buffers)");
  }
  return SPH_OK;
}

// user-order scatter of one field of every tank (each tank's live copy)
struct FieldSrc {
  const void* s[2][3];
  const uint32_t* id[2];
  int is_float, stride, off, comps;
};

__global__ void kb_scatter_field(BatchArgs A, FieldSrc f, double* __restrict__ out) {
  const WorkList* wl = A.wl_all;
  for_each_tile(wl, [&](int a, int first, int tile) {
    const int t = wl->tank[a];
    const Params& P = A.tP[t];
    const int par = A.tsc[t].par;
    const uint32_t* id = par ? f.id[1] : f.id[0];
    const int end = min(first + tile, P.n);
    for (int q = first + (int)threadIdx.x; q < end; q += blockDim.x) {
      const size_t k = (size_t)(P.foff + q);
      const size_t u = id[k];
      for (int c = 0; c < f.comps; ++c) {
        const void* src = par ? f.s[1][c] : f.s[0][c];
        const size_t e = k * f.stride + f.off;
        out[u * f.comps + c] =
            f.is_float ? (double)((const float*)src)[e] : ((const double*)src)[e];
      }
    }
  });
}

int scatter_out(sph_batch* b, FieldSrc f, double* host) {
  const int grid = b->A.tiles_max < 1 ? 1 : (b->A.tiles_max < b->L.blocks_stream ? b->A.tiles_max
                                                                               : b->L.blocks_stream);
  kb_scatter_field<<<grid, b->L.block_loop, 0, b->mem.stream>>>(b->A, f, b->B.io);
  CKB(cudaGetLastError());
  CKB(cudaMemcpyAsync(host, b->B.io, b->N * f.comps * sizeof(double), cudaMemcpyDeviceToHost,
                      b->mem.stream));
  CKB(cudaStreamSynchronize(b->mem.stream));
  return SPH_OK;
}

FieldSrc field_src(const void* a0, const void* a1, const void* a2, const void* b0,
                   const void* b1, const void* b2, const DevBuffers& B, int is_float, int stride,
                   int off, int comps) {
  FieldSrc f;
  f.s[0][0] = a0;
  f.s[0][1] = a1;
  f.s[0][2] = a2;
  f.s[1][0] = b0;
  f.s[1][1] = b1;
  f.s[1][2] = b2;
  f.id[0] = B.id[0];
  f.id[1] = B.id[1];
  f.is_float = is_float;
  f.stride = stride;
  f.off = off;
  f.comps = comps;
  return f;
}

}  // namespace

extern "C" {

int sph_create_batch(int n_tanks, const sph_tank* tanks, int precision,
                     const sph_allocator* alloc, void* stream, sph_batch** out) {
  if (!out) return SPH_E_INVALID;
  *out = nullptr;
  if (n_tanks < 1 || n_tanks > kMaxTanks || !tanks) return SPH_E_INVALID;
  if (precision != SPH_FP64 && precision != SPH_MIXED) return SPH_E_INVALID;
  if (alloc && (!alloc->alloc || !alloc->free)) return SPH_E_INVALID;
  const int dim = tanks[0].domain.dim;
  if (dim != 2 && dim != 3) return SPH_E_INVALID;
  std::vector<Params> P(n_tanks);
  std::vector<double> dps(n_tanks);
  long long total = 0;
  for (int t = 0; t < n_tanks; ++t) {
    const sph_tank& k = tanks[t];
    const sph_material& mat = k.material;
    if (k.domain.dim != dim) return SPH_E_INVALID;
    if (!(k.dp > 0) || !(k.h > 0) || !(mat.rho0 > 0) || !(mat.c0 > 0) || !(mat.mu >= 0) ||
        !(mat.U_ref > 0))
      return SPH_E_INVALID;
    const double cs = 2.0 * k.h;
    long long nc[3] = {1, 1, 1};
    long long ncell = 1;
    for (int a = 0; a < dim; ++a) {
      if (!(k.domain.hi[a] > k.domain.lo[a])) return SPH_E_INVALID;
      nc[a] = grid_cells(k.domain.lo[a], k.domain.hi[a], cs);
      if (nc[a] < 0) return SPH_E_INVALID;
      ncell *= nc[a];
      if (ncell > 0xfffffffll) return SPH_E_INVALID;
    }
    Params& p = P[t];
    memset(&p, 0, sizeof(p));
    p.dim = dim;
    p.nx = (int)nc[0];
    p.ny = (int)nc[1];
    p.nz = (int)nc[2];
    p.ncell = (uint32_t)ncell;
    for (int a = 0; a < 3; ++a) {
      p.lo[a] = a < dim ? k.domain.lo[a] : 0.0;
      p.g[a] = a < dim ? k.gravity[a] : 0.0;
    }
    p.cs = cs;
    p.h = k.h;
    p.r2max = 4.0 * k.h * k.h;
    p.rho0 = mat.rho0;
    p.c0 = mat.c0;
    p.c0sq = mat.c0 * mat.c0;
    p.mu = mat.mu;
    p.U_ref = mat.U_ref;
    p.V = dim == 2 ? k.dp * k.dp : k.dp * k.dp * k.dp;
    p.m = mat.rho0 * p.V;
    p.walpha = wendland_alpha(dim, k.h);
    p.sigma0 = lattice_sigma0(dim, k.dp, k.h, p.walpha);
    p.eps = 0.01 * k.h;
    p.diag = 0;
    p.use_list = 1;
    p.list_cap = dim == 3 ? 192 : 64;
    p.skin_max = 0.6 * k.h;
    p.variant = 0;
    p.cell_base = (uint32_t)total;
    total += ncell + 1;
    if (total >= (1ll << 31)) return SPH_E_INVALID;
    dps[t] = k.dp;
  }
  sph_batch* b = new sph_batch();
  b->T = n_tanks;
  b->dim = dim;
  b->precision = precision;
  b->P = P;
  b->dp = dps;
  b->total_cells = (uint32_t)total;
  if (alloc) {
    b->mem.alloc = *alloc;
    b->mem.has_alloc = true;
  }
  b->user_stream = (cudaStream_t)stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->L.sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->mem.stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = configure_sort_kernels();
  if (e != cudaSuccess) {
    int rc = cuda_err(b, e, "sph_create_batch");
    sph_batch_destroy(b);
    return rc;
  }
  b->L.radix_bits = 8;
  b->L.block_loop = 128;
  configure_launch(b);
  auto Af = [&](size_t bytes) { return b->mem.get(bytes, b->fixed_blocks); };
  const size_t ksize = precision == SPH_FP64 ? sizeof(stages::KC<double>) : sizeof(stages::KC<float>);
  b->A.tP = (const Params*)Af(sizeof(Params) * n_tanks);
  b->A.tK = Af(ksize * n_tanks);
  b->A.tsc = (DevScalars*)Af(sizeof(DevScalars) * n_tanks);
  // debug-build index checks record on tank 0's flags
  b->B.dbg_flags = b->A.tsc ? (int*)((char*)b->A.tsc + offsetof(DevScalars, flags)) : nullptr;
  b->A.wl_all = (WorkList*)Af(sizeof(WorkList));
  b->A.wl_adv = (WorkList*)Af(sizeof(WorkList));
  b->A.wl_wall = (WorkList*)Af(sizeof(WorkList));
  b->A.ntanks = n_tanks;
  b->B.cell_begin = (uint32_t*)Af((size_t)total * 4);
  b->B.wall_cb = (uint32_t*)Af((size_t)total * 4);
  b->B.digit_total = (uint32_t*)Af(((size_t)1 << kMaxRadixBits) * 4);
  // mixed path: each tank's cell-centre table of the record frame
  std::vector<int> ctab_off(n_tanks);
  size_t ctab_len = 0;
  for (int t = 0; t < n_tanks; ++t) {
    ctab_off[t] = (int)ctab_len;
    ctab_len += (size_t)(P[t].nx + P[t].ny + P[t].nz);
  }
  double* ctab = nullptr;
  int* ctab_off_dev = nullptr;
  if (precision == SPH_MIXED) {
    ctab = (double*)Af(ctab_len * 8);
    ctab_off_dev = (int*)Af((size_t)n_tanks * sizeof(int));
    if (!ctab || !ctab_off_dev) {
      sph_batch_destroy(b);
      return SPH_E_OOM;
    }
  }
  b->A.ctab = ctab;
  b->A.ctab_off = ctab_off_dev;
  if (!b->A.tP || !b->A.tK || !b->A.tsc || !b->A.wl_all || !b->A.wl_adv || !b->A.wl_wall ||
      !b->B.cell_begin || !b->B.wall_cb || !b->B.digit_total) {
    sph_batch_destroy(b);
    return SPH_E_OOM;
  }
  cudaStream_t s = b->mem.stream;
  e = cudaMemsetAsync(b->A.tsc, 0, sizeof(DevScalars) * n_tanks, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->B.cell_begin, 0, (size_t)total * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->B.wall_cb, 0, (size_t)total * 4, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->B.digit_total, 0, ((size_t)1 << kMaxRadixBits) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->A.wl_adv, 0, sizeof(WorkList), s);
  if (e == cudaSuccess && ctab) {
    e = cudaMemcpyAsync(ctab_off_dev, ctab_off.data(), sizeof(int) * n_tanks,
                        cudaMemcpyHostToDevice, s);
    for (int t = 0; t < n_tanks && e == cudaSuccess; ++t) {
      launch_centre_table(P[t], ctab + ctab_off[t], s);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // ctab_off is a host temporary
  }
  if (e != cudaSuccess) {
    int rc = cuda_err(b, e, "sph_create_batch");
    sph_batch_destroy(b);
    return rc;
  }
  int rc = upload_tables(b);
  if (!rc) rc = precision == SPH_FP64 ? upload_constants<double>(b) : upload_constants<float>(b);
  if (rc) {
    sph_batch_destroy(b);
    return rc;
  }
  *out = b;
  return SPH_OK;
}

int sph_batch_set_particles(sph_batch* b, int kind, const size_t* counts, const double* pos,
                            const double* vel, const double* rho) {
  TraceRange trace_("sph_batch_set_particles");
  if (!b) return SPH_E_INVALID;
  if (!counts) return set_err(b, SPH_E_INVALID, "counts is NULL");
  size_t total = 0;
  for (int t = 0; t < b->T; ++t) {
    if (counts[t] >= (1ull << 26)) return set_err(b, SPH_E_INVALID, "tank count too large");
    total += counts[t];
  }
  if (total >= (1ull << 26)) return set_err(b, SPH_E_INVALID, "at most 2^26 - 1 particles per kind");
  if (total > 0 && !pos) return set_err(b, SPH_E_INVALID, "pos is NULL");
  if (kind != SPH_FLUID && kind != SPH_WALL)
    return set_err(b, SPH_E_INVALID, "unknown particle kind");
  if (kind == SPH_WALL && rho) return set_err(b, SPH_E_INVALID, "wall particles take no density");
  const int d = b->dim;
  // prescribed (sliding) wall velocities: the walls read them only if one is nonzero
  bool moving = false;
  if (kind == SPH_WALL && vel) {
    for (size_t q = 0; q < total * (size_t)d; ++q) {
      if (!std::isfinite(vel[q])) return set_err(b, SPH_E_INVALID, "wall velocity is not finite");
      moving = moving || vel[q] != 0.0;
    }
  }
  cudaStream_t s = b->mem.stream;
  int rc = enter(b);
  if (rc) return rc;
  CKB(cudaStreamSynchronize(s));
  drop_graph(b);
  size_t off = 0;
  for (int t = 0; t < b->T; ++t) {
    if (kind == SPH_FLUID) {
      b->P[t].n = (int)counts[t];
      b->P[t].foff = (int)off;
    } else {
      b->P[t].nw = (int)counts[t];
      b->P[t].woff = (int)off;
      // every tank reads the (possibly zero) velocities of its walls: with
      // v_w = 0 the wall terms are bit-identical to those of walls at rest
      b->P[t].variant = moving ? (b->P[t].variant | kVariantMovingWall)
                               : (b->P[t].variant & ~kVariantMovingWall);
    }
    off += counts[t];
  }
  if (kind == SPH_FLUID) {
    b->N = total;
    rc = alloc_fluid(b, total);
    if (rc) {
      b->N = 0;
      b->fluid_set = false;
      return rc;
    }
  } else {
    b->NW = total;
  }
  configure_launch(b);
  rc = upload_tables(b);
  if (rc) return rc;
  DevBuffers& B = b->B;
  if (kind == SPH_FLUID) {
    const size_t n = total;
    if (n > 0) {
      CKB(cudaMemcpyAsync(B.io, pos, n * d * 8, cudaMemcpyHostToDevice, s));
      launch_deinterleave(B.io, (int)n, d, B.x[0], s);
      if (vel) {
        CKB(cudaMemcpyAsync(B.io, vel, n * d * 8, cudaMemcpyHostToDevice, s));
        launch_deinterleave(B.io, (int)n, d, B.v[0], s);
      } else {
        for (int k = 0; k < d; ++k) CKB(cudaMemsetAsync(B.v[0][k], 0, n * 8, s));
      }
      if (rho) {
        CKB(cudaMemcpyAsync(B.rho[0], rho, n * 8, cudaMemcpyHostToDevice, s));
      } else {
        // each tank's rest density (input marshalling of the defaults)
        std::vector<double> r(n);
        for (int t = 0; t < b->T; ++t)
          for (int q = 0; q < b->P[t].n; ++q) r[(size_t)b->P[t].foff + q] = b->P[t].rho0;
        CKB(cudaMemcpyAsync(B.rho[0], r.data(), n * 8, cudaMemcpyHostToDevice, s));
        CKB(cudaStreamSynchronize(s));
      }
      launch_init_fluid(B.rho[0], 0, 0.0, B.id[0], (int)n, s);
      CKB(cudaMemsetAsync(B.drho[0], 0, n * tsize(b), s));
      for (int k = 0; k < d; ++k) {
        CKB(cudaMemsetAsync(B.acc[k], 0, n * tsize(b), s));
        CKB(cudaMemsetAsync(B.aprior[k], 0, n * tsize(b), s));
      }
      CKB(cudaMemsetAsync(B.sigma, 0, n * tsize(b), s));
      CKB(cudaGetLastError());
    }
    CKB(cudaMemsetAsync(b->A.tsc, 0, sizeof(DevScalars) * b->T, s));
    if (b->precision == SPH_FP64)
      enqueue_batch_initial_sort_fp64(args(b), s);
    else
      enqueue_batch_initial_sort_mixed(args(b), s);
    const int grid = b->A.tiles_max < 1 ? 1 : (b->A.tiles_max < b->L.blocks_stream
                                                    ? b->A.tiles_max
                                                    : b->L.blocks_stream);
    launch_batch_vmax(b->A, b->B, grid, b->L.block_loop, s);
    CKB(cudaGetLastError());
    b->fluid_set = n > 0;
    CKB(cudaStreamSynchronize(s));
    return leave(b);
  }
  // walls
  b->mem.release(b->wall_blocks);
  const size_t n = total;
  B.wallP = B.wall_id = nullptr;
  B.wall_xyz = nullptr;
  B.wallI = nullptr;
  B.wall_vel = nullptr;
  if (n == 0) {
    CKB(cudaMemsetAsync(B.wall_cb, 0, (size_t)b->total_cells * 4, s));
    CKB(cudaStreamSynchronize(s));
    return leave(b);
  }
  auto Al = [&](size_t bytes) { return b->mem.get(bytes, b->wall_blocks); };
  const size_t ts = tsize(b);
  B.wallP = Al(n * (d == 3 ? 4 : 2) * ts);
  B.wall_id = (uint32_t*)Al(n * 4);
  B.wall_xyz = (double*)Al(n * 3 * 8);
  B.wallI = b->precision == SPH_MIXED ? Al(n * (d == 3 ? 16 : 8)) : nullptr;
  B.wall_vel = moving ? Al(n * (d == 3 ? 4 : 2) * ts) : nullptr;
  std::vector<Block> tmp;
  DevBuffers W = B;
  // staging: positions SoA (3 n), then the velocities SoA (3 n) when moving
  W.io = (double*)b->mem.get(n * (moving ? 6 : 3) * 8, tmp);
  for (int p = 0; p < 2; ++p) {
    W.keys[p] = (uint32_t*)b->mem.get(n * 4, tmp);
    W.vals[p] = (uint32_t*)b->mem.get(n * 4, tmp);
  }
  const size_t tiles = (n + kSortTile - 1) / kSortTile;
  W.tile_hist = (uint32_t*)b->mem.get(tiles * ((size_t)1 << kMaxRadixBits) * 4, tmp);
  const bool ok = B.wallP && B.wall_id && B.wall_xyz && W.io && W.keys[0] && W.keys[1] &&
                  W.vals[0] && W.vals[1] && W.tile_hist &&
                  (b->precision != SPH_MIXED || B.wallI) && (!moving || B.wall_vel);
  if (!ok) {
    b->mem.release(tmp);
    b->mem.release(b->wall_blocks);
    B.wall_vel = nullptr;
    for (int t = 0; t < b->T; ++t) {
      b->P[t].nw = 0;
      b->P[t].variant &= ~kVariantMovingWall;
    }
    b->NW = 0;
    upload_tables(b);
    return set_err(b, SPH_E_OOM, "device allocation failed (wall buffers)");
  }
  CKB(cudaMemcpyAsync(B.wall_xyz, pos, n * d * 8, cudaMemcpyHostToDevice, s));
  double* soa[3] = {W.io, W.io + n, W.io + 2 * n};
  if (d == 2) CKB(cudaMemsetAsync(W.io + 2 * n, 0, n * 8, s));
  launch_deinterleave(B.wall_xyz, (int)n, d, soa, s);
  if (moving) {
    // the AoS scratch is free again once the positions are deinterleaved
    CKB(cudaMemcpyAsync(B.wall_xyz, vel, n * d * 8, cudaMemcpyHostToDevice, s));
    double* vsoa[3] = {W.io + 3 * n, W.io + 4 * n, W.io + 5 * n};
    if (d == 2) CKB(cudaMemsetAsync(W.io + 5 * n, 0, n * 8, s));
    launch_deinterleave(B.wall_xyz, (int)n, d, vsoa, s);
  }
  BatchStageArgs a = args(b);
  a.B = W;
  if (b->precision == SPH_FP64)
    enqueue_batch_wall_setup_fp64(a, s);
  else
    enqueue_batch_wall_setup_mixed(a, s);
  CKB(cudaGetLastError());
  kb_lists_bad<<<(b->T + 255) / 256, 256, 0, s>>>(b->A.tsc, b->T);
  CKB(cudaGetLastError());
  CKB(cudaStreamSynchronize(s));
  b->mem.release(tmp);
  return leave(b);
}

int sph_batch_step(sph_batch* b, int n) {
  TraceRange trace_("sph_batch_step");
  if (!b) return SPH_E_INVALID;
  if (n < 0) return set_err(b, SPH_E_INVALID, "negative step count");
  if (!b->fluid_set) return set_err(b, SPH_E_STATE, "no fluid particles set");
  if (n == 0) return SPH_OK;
  int rc = enter(b);
  if (rc) return rc;
  cudaStream_t s = b->mem.stream;
  if (b->use_graph) {
    if (!b->graph_exec) {
      CKB(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      enqueue_step(b, s);
      cudaError_t e = cudaStreamEndCapture(s, &b->graph);
      if (e != cudaSuccess) {
        b->graph = nullptr;
        return cuda_err(b, e, "graph capture");
      }
      e = cudaGraphInstantiate(&b->graph_exec, b->graph, 0);
      if (e != cudaSuccess) {
        drop_graph(b);
        return cuda_err(b, e, "graph instantiate");
      }
    }
    for (int i = 0; i < n; ++i) CKB(cudaGraphLaunch(b->graph_exec, s));
  } else {
    for (int i = 0; i < n; ++i) enqueue_step(b, s);
    CKB(cudaGetLastError());
  }
  return leave(b);
}

int sph_batch_synchronize(sph_batch* b, double timeout_s) {
  if (!b) return SPH_E_INVALID;
  CKB(cudaEventRecord(b->ev_out, b->mem.stream));
  if (timeout_s > 0) {
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
      cudaError_t e = cudaEventQuery(b->ev_out);
      if (e == cudaSuccess) break;
      if (e != cudaErrorNotReady) return cuda_err(b, e, "sph_batch_synchronize");
      double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > timeout_s) return set_err(b, SPH_E_TIMEOUT, "queued work did not finish in time");
      std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
  }
  return sync_status(b);
}

int sph_batch_get_fields(sph_batch* b, unsigned mask, double* out) {
  TraceRange trace_("sph_batch_get_fields");
  if (!b || (!out && mask)) return SPH_E_INVALID;
  if (mask & ~0xffu) return set_err(b, SPH_E_INVALID, "unknown field bit");
  if (!b->fluid_set) return set_err(b, SPH_E_STATE, "no fluid particles set");
  int rc = enter(b);
  if (rc) return rc;
  std::vector<DevScalars> hs;
  rc = read_scalars(b, hs);
  if (rc) return rc;
  const int d = b->dim;
  const DevBuffers& B = b->B;
  const int isf = b->precision == SPH_MIXED;
  double* o = out;
  for (unsigned bit = 1; bit <= SPH_F_SIGMA; bit <<= 1) {
    if (!(mask & bit)) continue;
    FieldSrc f;
    switch (bit) {
      case SPH_F_POS:
        f = field_src(B.x[0][0], B.x[0][1], B.x[0][2], B.x[1][0], B.x[1][1], B.x[1][2], B, 0, 1,
                      0, d);
        break;
      case SPH_F_VEL:
        f = field_src(B.v[0][0], B.v[0][1], B.v[0][2], B.v[1][0], B.v[1][1], B.v[1][2], B, 0, 1,
                      0, d);
        break;
      case SPH_F_RHO:
        f = field_src(B.rho[0], 0, 0, B.rho[1], 0, 0, B, 0, 1, 0, 1);
        break;
      case SPH_F_P:
        // pressure of the last first half-step, kept in the records of buffer 0
        if (d == 3)
          f = field_src(B.rec[0], 0, 0, B.rec[0], 0, 0, B, isf, 8, 3, 1);
        else
          f = field_src(B.rec_s[0], 0, 0, B.rec_s[0], 0, 0, B, isf, 2, 0, 1);
        break;
      case SPH_F_DRHO:
        f = field_src(B.drho[0], 0, 0, B.drho[1], 0, 0, B, isf, 1, 0, 1);
        break;
      case SPH_F_ACC:
        f = field_src(B.acc[0], B.acc[1], B.acc[2], B.acc[0], B.acc[1], B.acc[2], B, isf, 1, 0, d);
        break;
      case SPH_F_APRIOR:
        f = field_src(B.aprior[0], B.aprior[1], B.aprior[2], B.aprior[0], B.aprior[1],
                      B.aprior[2], B, isf, 1, 0, d);
        break;
      default:  // SPH_F_SIGMA
        f = field_src(B.sigma, 0, 0, B.sigma, 0, 0, B, isf, 1, 0, 1);
        break;
    }
    rc = scatter_out(b, f, o);
    if (rc) return rc;
    o += b->N * f.comps;
  }
  rc = leave(b);
  if (rc) return rc;
  return flags_status(b, hs);
}

int sph_batch_get_scalars(sph_batch* b, double* t, double* dt_ad, double* dt_ac, long* n_ac,
                          long* n_adv) {
  if (!b) return SPH_E_INVALID;
  int rc = enter(b);
  if (rc) return rc;
  std::vector<DevScalars> hs;
  rc = read_scalars(b, hs);
  if (rc) return rc;
  for (int k = 0; k < b->T; ++k) {
    if (t) t[k] = hs[k].t;
    if (dt_ad) dt_ad[k] = hs[k].dt_ad;
    if (dt_ac) dt_ac[k] = hs[k].dt_ac;
    if (n_ac) n_ac[k] = (long)hs[k].n_ac;
    if (n_adv) n_adv[k] = (long)hs[k].n_adv;
  }
  rc = leave(b);
  if (rc) return rc;
  return flags_status(b, hs);
}

int sph_batch_debug_neighbour_state(sph_batch* b, int tank, uint32_t* keys, uint32_t* ids,
                                    uint32_t* cell_begin) {
  if (!b) return SPH_E_INVALID;
  if (tank < 0 || tank >= b->T) return set_err(b, SPH_E_INVALID, "tank out of range");
  if (!b->fluid_set) return set_err(b, SPH_E_STATE, "no fluid particles set");
  int rc = enter(b);
  if (rc) return rc;
  std::vector<DevScalars> hs;
  rc = read_scalars(b, hs);
  if (rc) return rc;
  const Params& P = b->P[tank];
  const size_t n = (size_t)P.n;
  cudaStream_t s = b->mem.stream;
  if (keys && n)
    CKB(cudaMemcpyAsync(keys, b->A.bkey + P.foff, n * 4, cudaMemcpyDeviceToHost, s));
  if (ids && n)
    CKB(cudaMemcpyAsync(ids, b->B.id[hs[tank].par] + P.foff, n * 4, cudaMemcpyDeviceToHost, s));
  if (cell_begin)
    CKB(cudaMemcpyAsync(cell_begin, b->B.cell_begin + P.cell_base, ((size_t)P.ncell + 1) * 4,
                        cudaMemcpyDeviceToHost, s));
  CKB(cudaStreamSynchronize(s));
  // the tank's own numbering: slots and user indices start at its first slot
  if (ids)
    for (size_t q = 0; q < n; ++q) ids[q] -= (uint32_t)P.foff;
  if (cell_begin)
    for (size_t c = 0; c <= P.ncell; ++c) cell_begin[c] -= (uint32_t)P.foff;
  rc = leave(b);
  if (rc) return rc;
  return flags_status(b, hs);
}

size_t sph_batch_count(const sph_batch* b, int kind) {
  if (!b) return 0;
  return kind == SPH_WALL ? b->NW : b->N;
}

int sph_batch_tank_count(const sph_batch* b) { return b ? b->T : 0; }

size_t sph_batch_cell_count(const sph_batch* b, int tank) {
  if (!b || tank < 0 || tank >= b->T) return 0;
  return b->P[tank].ncell;
}

int sph_batch_profile_stages(sph_batch* b, int n, double* ms, long* rebuilds) {
  if (!b || !ms || n < 0) return SPH_E_INVALID;
  if (!b->fluid_set) return set_err(b, SPH_E_STATE, "no fluid particles set");
  int rc = enter(b);
  if (rc) return rc;
  std::vector<DevScalars> before, after;
  rc = read_scalars(b, before);
  if (rc) return rc;
  cudaEvent_t ev[kStages + 1];
  for (int k = 0; k <= kStages; ++k) CKB(cudaEventCreate(&ev[k]));
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    enqueue_step(b, b->mem.stream, ev);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[kStages]);
    for (int k = 0; k < kStages && e == cudaSuccess; ++k) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
      ms[k] += t;
    }
  }
  for (int k = 0; k <= kStages; ++k) cudaEventDestroy(ev[k]);
  if (e != cudaSuccess) return cuda_err(b, e, "sph_batch_profile_stages");
  rc = read_scalars(b, after);
  if (rc) return rc;
  if (rebuilds) {
    long r = 0;
    for (int t = 0; t < b->T; ++t) r += (long)(after[t].n_adv - before[t].n_adv);
    *rebuilds = r;
  }
  rc = leave(b);
  if (rc) return rc;
  return flags_status(b, after);
}

long sph_batch_kernels_per_step(const sph_batch* cb) {
  if (!cb) return -1;
  sph_batch* b = const_cast<sph_batch*>(cb);
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(b->mem.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return -1;
  enqueue_step(b, b->mem.stream);
  if (cudaStreamEndCapture(b->mem.stream, &g) != cudaSuccess || !g) return -1;
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

int sph_batch_set_option(sph_batch* b, int option, long value) {
  if (!b) return SPH_E_INVALID;
  int rc = SPH_OK;
  const int old_list = b->P[0].use_list;
  switch (option) {
    case SPH_OPT_RECORD_DIAGNOSTICS:
      for (auto& p : b->P) p.diag = value ? 1 : 0;
      break;
    case SPH_OPT_USE_GRAPH:
      b->use_graph = value != 0;
      break;
    case SPH_OPT_BLOCK:
      if (value < 64 || value > 256 || value % 32)
        return set_err(b, SPH_E_INVALID, "block size must be 64..256, a multiple of 32");
      b->L.block_loop = (int)value;
      configure_launch(b);
      break;
    case SPH_OPT_NEIGHBOUR_LIST:
      for (auto& p : b->P) p.use_list = value ? 1 : 0;
      break;
    case SPH_OPT_RADIX_BITS:
      if (value < 4 || value > kMaxRadixBits)
        return set_err(b, SPH_E_INVALID, "radix bits must be 4..11");
      b->L.radix_bits = (int)value;
      configure_launch(b);
      break;
    case SPH_OPT_DENSITY_RIEMANN:
      for (auto& p : b->P)
        p.variant = value ? (p.variant & ~kVariantNoRiemann) : (p.variant | kVariantNoRiemann);
      break;
    case SPH_OPT_REINIT_BLENDED:
      for (auto& p : b->P)
        p.variant = value ? (p.variant | kVariantBlended) : (p.variant & ~kVariantBlended);
      break;
    case SPH_OPT_TRANSPORT_CORRECTION:
      for (auto& p : b->P)
        p.variant = value ? (p.variant | kVariantTransport) : (p.variant & ~kVariantTransport);
      break;
    default:
      return set_err(b, SPH_E_INVALID, "unknown option");
  }
  rc = enter(b);
  if (rc) return rc;
  CKB(cudaStreamSynchronize(b->mem.stream));
  drop_graph(b);
  rc = upload_tables(b);
  if (!rc)
    rc = b->precision == SPH_FP64 ? upload_constants<double>(b) : upload_constants<float>(b);
  if (rc) return rc;
  if (b->P[0].use_list && !old_list) {
    // no list was built at the tanks' last rebuilds: direct search until the next ones
    std::vector<DevScalars> hs;
    rc = read_scalars(b, hs);
    if (rc) return rc;
    for (auto& h : hs) h.list_bad = 1;
    CKB(cudaMemcpyAsync(b->A.tsc, hs.data(), sizeof(DevScalars) * b->T, cudaMemcpyHostToDevice,
                        b->mem.stream));
    CKB(cudaStreamSynchronize(b->mem.stream));
  }
  return leave(b);
}

int sph_batch_autotune(sph_batch* b, int steps_per_trial, sph_tuning* best) {
  TraceRange trace_("sph_batch_autotune");
  if (!b || !best || steps_per_trial < 1) return SPH_E_INVALID;
  if (!b->fluid_set) return set_err(b, SPH_E_STATE, "no fluid particles set");
  int rc = enter(b);
  if (rc) return rc;
  cudaStream_t s = b->mem.stream;
  CKB(cudaStreamSynchronize(s));
  Snapshot snap;
  if (!snap.take(b->mem, {&b->fluid_blocks, &b->wall_blocks, &b->fixed_blocks}))
    return set_err(b, SPH_E_OOM, "device allocation failed (autotuner snapshot)");
  const LaunchCfg L0 = b->L;
  const std::vector<Params> P0 = b->P;
  const int sorted0 = b->B.sorted_buf;
  const bool graph0 = b->use_graph;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto reset = [&]() -> int {
    drop_graph(b);
    if (snap.restore(s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
      return SPH_E_CUDA;
    b->L = L0;
    b->P = P0;
    b->B.sorted_buf = sorted0;
    b->use_graph = true;
    return upload_tables(b);
  };
  auto apply = [&](const sph_tuning& t) -> int {
    int r = sph_batch_set_option(b, SPH_OPT_BLOCK, t.block);
    if (!r) r = sph_batch_set_option(b, SPH_OPT_RADIX_BITS, t.radix_bits);
    if (!r) r = sph_batch_set_option(b, SPH_OPT_NEIGHBOUR_LIST, t.neighbour_list);
    return r;
  };
  auto trial = [&](const sph_tuning& t) -> double {
    double bestms = -1.0;
    for (int rep = 0; rep < 2; ++rep) {
      if (reset() || apply(t)) return -1.0;
      if (cudaEventRecord(e0, b->user_stream) != cudaSuccess) return -1.0;
      if (sph_batch_step(b, steps_per_trial)) return -1.0;
      if (cudaEventRecord(e1, b->user_stream) != cudaSuccess) return -1.0;
      if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0;
      const double per = ms / steps_per_trial;
      if (bestms < 0 || per < bestms) bestms = per;
    }
    return bestms;
  };
  sph_tuning start{L0.block_loop, L0.radix_bits, P0[0].use_list, 0, 0.0};
  sph_tuning found = start;
  int search = e == cudaSuccess ? tune_search(start, trial, &found) : -1;
  rc = reset();
  if (!rc) rc = apply(search == 0 ? found : start);
  b->use_graph = graph0;
  snap.drop(b->mem);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (search != 0)
    return rc ? rc : set_err(b, SPH_E_CUDA, "autotuner trial failed: " + b->err);
  if (rc) return rc;
  *best = found;
  return leave(b);
}

const char* sph_batch_last_error(const sph_batch* b) { return b ? b->err.c_str() : "null batch"; }

void sph_batch_destroy(sph_batch* b) {
  if (!b) return;
  if (b->mem.stream) cudaStreamSynchronize(b->mem.stream);
  drop_graph(b);
  b->mem.release(b->fluid_blocks);
  b->mem.release(b->wall_blocks);
  b->mem.release(b->fixed_blocks);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->mem.stream) cudaStreamDestroy(b->mem.stream);
  delete b;
}

}  // extern "C"
