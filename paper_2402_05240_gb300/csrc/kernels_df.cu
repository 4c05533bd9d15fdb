// Instantiation of the step kernels for the FP64-accurate step computed in
// double-float arithmetic on the FP32 pipes.
#include "mhd_kernels.cuh"

namespace mhd {
template struct Launch<df>;
}  // namespace mhd
