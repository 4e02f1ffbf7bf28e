// 3D instantiations of the reverse-pass kernels (float, double).
#include "sph_adjoint_impl.cuh"

namespace sph {
SPH_INSTANTIATE_ADJOINT(3, float)
SPH_INSTANTIATE_ADJOINT(3, double)
}  // namespace sph
