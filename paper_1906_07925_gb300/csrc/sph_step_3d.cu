// 3D instantiations of the relaxation-step kernels (float split precision, double).
#include "sph_step_impl.cuh"

namespace sph {
SPH_INSTANTIATE_STEP(3, float)
SPH_INSTANTIATE_STEP(3, double)
template cudaError_t prepare_staged_pass<3>();
}  // namespace sph
