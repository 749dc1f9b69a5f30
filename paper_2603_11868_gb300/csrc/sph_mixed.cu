// Mixed path: pair interactions in float with float sums over float cell-local
// offsets; positions, keys, velocity and density state in double.
#include "sph_stages.cuh"

namespace sphgb {

void enqueue_step_mixed(const StageArgs& a, cudaStream_t s, cudaEvent_t* ev) {
  if (a.P.dim == 2)
    stages::enqueue_step_t<2, float>(a, s, ev);
  else
    stages::enqueue_step_t<3, float>(a, s, ev);
}

void enqueue_advection_mixed(const StageArgs& a, cudaStream_t s) {
  if (a.P.dim == 2)
    stages::enqueue_advection_t<2, float>(a, s);
  else
    stages::enqueue_advection_t<3, float>(a, s);
}

void enqueue_acoustic_mixed(const StageArgs& a, cudaStream_t s) {
  if (a.P.dim == 2)
    stages::enqueue_acoustic_t<2, float>(a, s);
  else
    stages::enqueue_acoustic_t<3, float>(a, s);
}

void enqueue_initial_sort_mixed(const StageArgs& a, cudaStream_t s) {
  if (a.P.dim == 2)
    stages::enqueue_initial_sort_t<2, float>(a, s);
  else
    stages::enqueue_initial_sort_t<3, float>(a, s);
}

void enqueue_wall_setup_mixed(const StageArgs& a, cudaStream_t s) {
  if (a.P.dim == 2)
    stages::enqueue_wall_setup_t<2, float>(a, s);
  else
    stages::enqueue_wall_setup_t<3, float>(a, s);
}

}  // namespace sphgb
