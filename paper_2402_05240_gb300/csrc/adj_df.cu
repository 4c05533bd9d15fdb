// Instantiation of the adjoint kernels for the double-float step.
#include "mhd_adjoint_kernels.cuh"

namespace mhd {
template struct AdjLaunch<df>;
}  // namespace mhd
