// Mixed path of the batched stages (instantiations).
#include "sph_batch_stages.cuh"

namespace sphgb {

void enqueue_batch_step_mixed(const BatchStageArgs& a, cudaStream_t s, cudaEvent_t* ev) {
  if (a.dim == 2)
    stages::enqueue_batch_step_t<2, float>(a, s, ev);
  else
    stages::enqueue_batch_step_t<3, float>(a, s, ev);
}

void enqueue_batch_initial_sort_mixed(const BatchStageArgs& a, cudaStream_t s) {
  if (a.dim == 2)
    stages::enqueue_batch_initial_sort_t<2, float>(a, s);
  else
    stages::enqueue_batch_initial_sort_t<3, float>(a, s);
}

void enqueue_batch_wall_setup_mixed(const BatchStageArgs& a, cudaStream_t s) {
  if (a.dim == 2)
    stages::enqueue_batch_wall_setup_t<2, float>(a, s);
  else
    stages::enqueue_batch_wall_setup_t<3, float>(a, s);
}

}  // namespace sphgb
