// Mixed path: pair interactions in float with float sums over float cell-local
// offsets; positions, keys, velocity and density state in double.
#include "sph_stages.cuh"

namespace sphgb {

namespace {
__global__ void k_centre_table(Params P, double* tab) {
  const int total = P.nx + P.ny + P.nz;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int k = t < P.nx ? 0 : (t < P.nx + P.ny ? 1 : 2);
    const int c = k == 0 ? t : (k == 1 ? t - P.nx : t - P.nx - P.ny);
    tab[t] = stages::Local<float>::centre(P, k, c);
  }
}
}  // namespace

void launch_centre_table(const Params& P, double* tab, cudaStream_t s) {
  const int total = P.nx + P.ny + P.nz;
  k_centre_table<<<(total + 255) / 256, 256, 0, s>>>(P, tab);
}

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

void enqueue_wall_rebin_mixed(const StageArgs& a, cudaStream_t s, int at_rebuild) {
  const int when = at_rebuild ? stages::kBinAtRebuild : stages::kBinNow;
  if (a.P.dim == 2)
    stages::enqueue_wall_rebin_t<2, float>(a, s, 0, when);
  else
    stages::enqueue_wall_rebin_t<3, float>(a, s, 0, when);
}

void enqueue_units_mixed(const StageArgs& a, cudaStream_t s) {
  if (a.P.dim == 3) stages::enqueue_units<3, float>(a, s, 0);
}

void enqueue_restore_lists_mixed(const StageArgs& a, cudaStream_t s) {
  if (a.P.dim == 2)
    stages::enqueue_restore_lists_t<2, float>(a, s);
  else
    stages::enqueue_restore_lists_t<3, float>(a, s);
}

}  // namespace sphgb
