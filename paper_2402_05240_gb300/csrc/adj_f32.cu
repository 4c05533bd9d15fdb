// Instantiation of the adjoint kernels for the FP32-bulk step.
#include "mhd_adjoint_kernels.cuh"

namespace mhd {
template struct AdjLaunch<float>;
}  // namespace mhd
