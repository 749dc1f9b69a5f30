// Plain FP64 path of the batched stages (instantiations).
#include "sph_batch_stages.cuh"

namespace sphgb {

void enqueue_batch_step_fp64(const BatchStageArgs& a, cudaStream_t s, cudaEvent_t* ev) {
  if (a.dim == 2)
    stages::enqueue_batch_step_t<2, double>(a, s, ev);
  else
    stages::enqueue_batch_step_t<3, double>(a, s, ev);
}

void enqueue_batch_initial_sort_fp64(const BatchStageArgs& a, cudaStream_t s) {
  if (a.dim == 2)
    stages::enqueue_batch_initial_sort_t<2, double>(a, s);
  else
    stages::enqueue_batch_initial_sort_t<3, double>(a, s);
}

void enqueue_batch_wall_setup_fp64(const BatchStageArgs& a, cudaStream_t s) {
  if (a.dim == 2)
    stages::enqueue_batch_wall_setup_t<2, double>(a, s);
  else
    stages::enqueue_batch_wall_setup_t<3, double>(a, s);
}

}  // namespace sphgb
