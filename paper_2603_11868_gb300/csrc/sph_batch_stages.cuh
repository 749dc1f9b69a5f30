// Batched stages: many independent tanks advance together, one persistent
// launch per stage.  Each launch walks a work list (sph_internal.cuh) tile by
// tile and runs the one-tank bodies of sph_stages.cuh on the tile's slot range
// with the tile's tank parameters, constants and schedule, so a tank of the
// batch computes exactly what it computes alone.  The stages that follow a
// rebuild (keys, sort, reorder, offsets, lists, density summation, viscous
// force) walk only the tanks that begin an advection step in this acoustic
// step; the acoustic stages walk every tank.
#pragma once

#include <stddef.h>

#include "sph_stages.cuh"

namespace sphgb {
namespace stages {

// f(tank, its Params, first slot of this thread, end of the tile) per tile
template <class F>
__device__ __forceinline__ void for_each_tank_tile(const BatchArgs& A, const WorkList* wl, F&& f) {
  for_each_tile(wl, [&](int a, int off, int tile) {
    const int t = wl->tank[a];
    const Params P = A.tP[t];
    const int i0 = P.foff + off;
    const int i1 = min(i0 + tile, P.foff + P.n);
    f(t, P, i0 + (int)threadIdx.x, i1);
  });
}

template <class T>
__device__ __forceinline__ KC<T> tank_kc(const BatchArgs& A, int t) {
  return ((const KC<T>*)A.tK)[t];
}

// the shared arrays with tank t's cell-centre table selected
__device__ __forceinline__ DevBuffers tank_buffers(const BatchArgs& A, const DevBuffers& B, int t) {
  DevBuffers Bt = B;
  Bt.ctab = A.ctab ? A.ctab + A.ctab_off[t] : nullptr;
  return Bt;
}

// Reorder of the listed tanks: compacted sorted slot cbase + q of a tank
// fills its slot foff + q from the slot named by the sorted value.
template <int D, class T>
__global__ void kb_reorder(BatchArgs A, DevBuffers B, const WorkList* wl) {
  const uint32_t* __restrict__ perm = B.vals[B.sorted_buf];
  const uint32_t* __restrict__ keys = B.keys[B.sorted_buf];
  for_each_tile(wl, [&](int a, int off, int tile) {
    const int t = wl->tank[a];
    const Params P = A.tP[t];
    const int par = A.tsc[t].par;
    const Live<T> S = live<T>(B, par), Dd = live<T>(B, par ^ 1);
    const DevBuffers Bt = tank_buffers(A, B, t);
    const int base = wl->cbase[a];
    const int end = min(off + tile, P.n);
    const BudgetArgs ba = budget_args(P, A.tsc[t]);
    for (int q = off + (int)threadIdx.x; q < end; q += blockDim.x) {
      const uint32_t key = keys[base + q] - P.cell_base;
      const int k = P.foff + q;
      A.bkey[k] = key;
      reorder_slot<D, T>(P, Bt, S, Dd, k, perm[base + q], key, ba);
    }
  });
}

template <int D, class T>
__global__ void kb_wall_gather(BatchArgs A, DevBuffers B, const double* __restrict__ ux,
                               const double* __restrict__ uy, const double* __restrict__ uz,
                               double* wx, double* wy, double* wz, const double* uv) {
  const uint32_t* __restrict__ perm = B.vals[B.sorted_buf];
  const uint32_t* __restrict__ keys = B.keys[B.sorted_buf];
  const WorkList* wl = A.wl_wall;
  for_each_tile(wl, [&](int a, int off, int tile) {
    const int t = wl->tank[a];
    const Params P = A.tP[t];
    const int base = wl->cbase[a];
    const int end = min(off + tile, P.nw);
    for (int q = off + (int)threadIdx.x; q < end; q += blockDim.x)
      wall_slot<D, T>(P, B, ux, uy, uz, wx, wy, wz, uv, (size_t)A.nw_total, P.woff + q,
                      perm[base + q], keys[base + q] - P.cell_base);
  });
}

template <int D, class T>
__global__ void __launch_bounds__(256, kMinBlocks<T>) kb_build_lists(BatchArgs A, DevBuffers B,
                                                                     const WorkList* wl) {
  for_each_tank_tile(A, wl, [&](int t, const Params& P, int i, int end) {
    if (P.use_list)
      build_lists_range<D, T>(P, B, tank_kc<T>(A, t), A.tsc + t, i, end, blockDim.x);
  });
}

template <int D, class T>
__global__ void __launch_bounds__(256, kMinBlocks<T>) kb_density_summation(BatchArgs A,
                                                                           DevBuffers B,
                                                                           const WorkList* wl) {
  for_each_tank_tile(A, wl, [&](int t, const Params& P, int i, int end) {
    if constexpr (Local<T>::kLocal)
      density_summation_fx_range<D>(P, B, A.tsc + t, i, end, blockDim.x);
    else
      density_summation_range<D, T>(P, B, tank_kc<T>(A, t), A.tsc + t, i, end, blockDim.x);
  });
}

template <int D, class T>
__global__ void __launch_bounds__(256, kMinBlocks<T>) kb_transport(BatchArgs A, DevBuffers B,
                                                                   const WorkList* wl) {
  __shared__ ShiftTable tab;
  if constexpr (Local<T>::kLocal) fill_shift_table(tab);
  for_each_tank_tile(A, wl, [&](int t, const Params& P, int i, int end) {
    if (P.variant & kVariantTransport)
      transport_range<D, T>(P, B, tank_kc<T>(A, t), A.tsc + t, i, end, blockDim.x, &tab);
  });
}

template <int D, class T>
__global__ void kb_transport_apply(BatchArgs A, DevBuffers B, const WorkList* wl) {
  for_each_tank_tile(A, wl, [&](int t, const Params& P, int i, int end) {
    if (P.variant & kVariantTransport)
      transport_apply_range<D, T>(P, tank_buffers(A, B, t), A.tsc + t, i, end, blockDim.x);
  });
}

template <int D, class T>
__global__ void __launch_bounds__(256, kMinBlocks<T>) kb_viscous(BatchArgs A, DevBuffers B,
                                                                 const WorkList* wl) {
  __shared__ ShiftTable tab;
  if constexpr (Local<T>::kLocal && !kShiftBits<D>) fill_shift_table(tab);
  for_each_tank_tile(A, wl, [&](int t, const Params& P, int i, int end) {
    viscous_range<D, T>(P, B, tank_kc<T>(A, t), A.tsc + t, i, end, blockDim.x, &tab);
  });
}

template <int D, class T>
__global__ void kb_half1(BatchArgs A, DevBuffers B, const WorkList* wl) {
  for_each_tank_tile(A, wl, [&](int t, const Params& P, int i, int end) {
    half1_range<D, T>(P, tank_buffers(A, B, t), A.tsc + t, i, end, blockDim.x);
  });
}

template <int D, class T, bool kWallVel>
__global__ void __launch_bounds__(256, kMinBlocksP<D, T>) kb_pressure(BatchArgs A, DevBuffers B,
                                                                  const WorkList* wl) {
  __shared__ ShiftTable tab;
  if constexpr (Local<T>::kLocal && !kShiftBits<D>) fill_shift_table(tab);
  for_each_tank_tile(A, wl, [&](int t, const Params& P, int i, int end) {
    pressure_range<D, T, kWallVel>(P, tank_buffers(A, B, t), tank_kc<T>(A, t), A.tsc + t, i, end,
                         blockDim.x, &tab);
  });
}

template <int D, class T, bool kWallVel>
__global__ void __launch_bounds__(256, kMinBlocksP<D, T>) kb_density_relax(BatchArgs A, DevBuffers B,
                                                                       const WorkList* wl) {
  __shared__ ShiftTable tab;
  if constexpr (Local<T>::kLocal && !kShiftBits<D>) fill_shift_table(tab);
  for_each_tank_tile(A, wl, [&](int t, const Params& P, int i, int end) {
    density_relax_range<D, T, kWallVel>(P, B, tank_kc<T>(A, t), A.tsc + t, i, end, blockDim.x,
                                       &tab);
  });
}

// ---------------------------------------------------------------------------
inline const int* wl_count_ptr(const WorkList* wl) {
  return (const int*)((const char*)wl + offsetof(WorkList, m));
}

inline int clamp_grid(int units, int cap) { return units < 1 ? 1 : (units < cap ? units : cap); }

// Rebuild of the tanks in wl_adv: keys -> one sort of their compacted slots ->
// reorder -> offsets (which also flip each rebuilt tank's live copy).
template <int D, class T>
void enqueue_batch_rebuild(const BatchStageArgs& a, cudaStream_t s, cudaEvent_t* ev) {
  const BatchArgs& A = a.A;
  const LaunchCfg& L = a.L;
  DevBuffers B = a.B;
  const int blk = L.block_loop;
  const int grid = clamp_grid(A.tiles_max, L.blocks_loop);
  uint32_t* keys[2] = {B.keys[0], B.keys[1]};
  uint32_t* vals[2] = {B.vals[0], B.vals[1]};
  mark(ev, kStageKeys, s);
  launch_batch_cell_keys(A, A.wl_adv, 0, B.x, keys[0], vals[0], B.digit_total,
                         1 << L.radix_bits, grid, blk, s);
  mark(ev, kStageSort, s);
  B.sorted_buf = launch_radix_sort_dev(L, keys, vals, A.n_total, B.tile_hist, B.digit_total,
                                       wl_count_ptr(A.wl_adv), s);
  mark(ev, kStageReorder, s);
  kb_reorder<D, T><<<grid, blk, 0, s>>>(A, B, A.wl_adv);
  mark(ev, kStageOffsets, s);
  launch_batch_cell_offsets(A, A.wl_adv, 0, clamp_grid(A.chunks_max, L.sms * 8), B.keys[B.sorted_buf],
                            B.cell_begin, 1, s);
}

template <int D, class T>
void enqueue_batch_step_t(const BatchStageArgs& a, cudaStream_t s, cudaEvent_t* ev) {
  const BatchArgs& A = a.A;
  const LaunchCfg& L = a.L;
  const DevBuffers& B = a.B;
  const int blk = L.block_loop;
  const int grid = clamp_grid(A.tiles_max, L.blocks_loop);
  mark(ev, kStageControl, s);
  launch_batch_control(A, blk, 0, s);
  enqueue_batch_rebuild<D, T>(a, s, ev);
  mark(ev, kStageDensitySum, s);
  kb_build_lists<D, T><<<grid, blk, 0, s>>>(A, B, A.wl_adv);
  kb_density_summation<D, T><<<grid, blk, 0, s>>>(A, B, A.wl_adv);
  if (a.variants & kVariantTransport) {
    kb_transport<D, T><<<grid, blk, 0, s>>>(A, B, A.wl_adv);
    kb_transport_apply<D, T><<<grid, blk, 0, s>>>(A, B, A.wl_adv);
  }
  mark(ev, kStageViscous, s);
  kb_viscous<D, T><<<grid, blk, 0, s>>>(A, B, A.wl_adv);
  mark(ev, kStageHalf1, s);
  kb_half1<D, T><<<grid, blk, 0, s>>>(A, B, A.wl_all);
  mark(ev, kStagePressure, s);
  const bool wall_vel = wall_vel_code<D>(a.variants);
  if (wall_vel)
    kb_pressure<D, T, true><<<grid, blk, 0, s>>>(A, B, A.wl_all);
  else
    kb_pressure<D, T, false><<<grid, blk, 0, s>>>(A, B, A.wl_all);
  mark(ev, kStageDensityRelax, s);
  if (wall_vel)
    kb_density_relax<D, T, true><<<grid, blk, 0, s>>>(A, B, A.wl_all);
  else
    kb_density_relax<D, T, false><<<grid, blk, 0, s>>>(A, B, A.wl_all);
  mark(ev, kStages, s);
}

template <int D, class T>
void enqueue_batch_initial_sort_t(const BatchStageArgs& a, cudaStream_t s) {
  launch_batch_control(a.A, a.L.block_loop, 1, s);
  enqueue_batch_rebuild<D, T>(a, s, nullptr);
}

template <int D, class T>
void enqueue_batch_wall_setup_t(const BatchStageArgs& a, cudaStream_t s) {
  const BatchArgs& A = a.A;
  const LaunchCfg& L = a.L;
  DevBuffers B = a.B;
  const size_t nw = (size_t)A.nw_total;
  double* io[2][3] = {{B.io, B.io + nw, B.io + 2 * nw}, {B.io, B.io + nw, B.io + 2 * nw}};
  double* wx = B.wall_xyz;
  double* wy = wx + nw;
  double* wz = wy + nw;
  uint32_t* keys[2] = {B.keys[0], B.keys[1]};
  uint32_t* vals[2] = {B.vals[0], B.vals[1]};
  const int wtiles = (int)((nw + 255) / 256) + A.ntanks;
  launch_batch_cell_keys(A, A.wl_wall, 1, io, keys[0], vals[0], B.digit_total,
                         1 << L.radix_bits, clamp_grid(wtiles, L.blocks_stream), 256, s);
  B.sorted_buf = launch_radix_sort(L, keys, vals, A.nw_total, B.tile_hist, B.digit_total,
                                   nullptr, 0, s);
  // velocity staging after the positions: io + 3 nw (x | y | z)
  const double* uv = B.wall_vel ? B.io + 3 * nw : nullptr;
  kb_wall_gather<D, T><<<clamp_grid(wtiles, L.blocks_stream), 256, 0, s>>>(
      A, B, io[0][0], io[0][1], io[0][2], wx, wy, wz, uv);
  launch_batch_cell_offsets(A, A.wl_wall, 1, clamp_grid(A.chunks_max, L.sms * 8),
                            B.keys[B.sorted_buf], B.wall_cb, 0, s);
}

}  // namespace stages
}  // namespace sphgb
