// FP64 path: every stage in double precision (records hold absolute positions).
#include "sph_stages.cuh"

namespace sphgb {

void enqueue_step_fp64(const StageArgs& a, cudaStream_t s, cudaEvent_t* ev) {
  if (a.P.dim == 2)
    stages::enqueue_step_t<2, double>(a, s, ev);
  else
    stages::enqueue_step_t<3, double>(a, s, ev);
}

void enqueue_advection_fp64(const StageArgs& a, cudaStream_t s) {
  if (a.P.dim == 2)
    stages::enqueue_advection_t<2, double>(a, s);
  else
    stages::enqueue_advection_t<3, double>(a, s);
}

void enqueue_acoustic_fp64(const StageArgs& a, cudaStream_t s) {
  if (a.P.dim == 2)
    stages::enqueue_acoustic_t<2, double>(a, s);
  else
    stages::enqueue_acoustic_t<3, double>(a, s);
}

void enqueue_initial_sort_fp64(const StageArgs& a, cudaStream_t s) {
  if (a.P.dim == 2)
    stages::enqueue_initial_sort_t<2, double>(a, s);
  else
    stages::enqueue_initial_sort_t<3, double>(a, s);
}

void enqueue_wall_setup_fp64(const StageArgs& a, cudaStream_t s) {
  if (a.P.dim == 2)
    stages::enqueue_wall_setup_t<2, double>(a, s);
  else
    stages::enqueue_wall_setup_t<3, double>(a, s);
}

void enqueue_wall_rebin_fp64(const StageArgs& a, cudaStream_t s, int at_rebuild) {
  const int when = at_rebuild ? stages::kBinAtRebuild : stages::kBinNow;
  if (a.P.dim == 2)
    stages::enqueue_wall_rebin_t<2, double>(a, s, 0, when);
  else
    stages::enqueue_wall_rebin_t<3, double>(a, s, 0, when);
}

void enqueue_restore_lists_fp64(const StageArgs& a, cudaStream_t s) {
  if (a.P.dim == 2)
    stages::enqueue_restore_lists_t<2, double>(a, s);
  else
    stages::enqueue_restore_lists_t<3, double>(a, s);
}

}  // namespace sphgb
