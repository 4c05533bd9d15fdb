// Instantiation of the step kernels for the FP32-bulk step.
#include "mhd_kernels.cuh"

namespace mhd {
template struct Launch<float>;
}  // namespace mhd
