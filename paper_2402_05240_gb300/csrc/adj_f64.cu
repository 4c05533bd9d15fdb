// Instantiation of the adjoint kernels for the FP64 step.
#include "mhd_adjoint_kernels.cuh"

namespace mhd {
template struct AdjLaunch<double>;
}  // namespace mhd
