// 2D instantiations of the relaxation-step kernels (float split precision, double).
#include "sph_step_impl.cuh"

namespace sph {
SPH_INSTANTIATE_STEP(2, float)
SPH_INSTANTIATE_STEP(2, double)
template cudaError_t prepare_staged_pass<2>();
}  // namespace sph
