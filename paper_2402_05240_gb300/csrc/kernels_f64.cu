// Instantiation of the step kernels for the FP64 step.
#define MHD_SCALAR_KERNELS  // dt and diagnostics kernels live in this unit only
#include "mhd_kernels.cuh"

namespace mhd {
template struct Launch<double>;

void launch_set_dt(const Grid& g, double* dt_cur, double value, cudaStream_t s) {
  k_set_dt<<<1, 1, 0, s>>>(g, dt_cur, value);
}
void launch_finish_dt(const Grid& g, unsigned long long* dtbits, double* dt_cur, double* dt_log, int step,
                      unsigned* flags, double t_end, cudaStream_t s) {
  k_finish_dt<<<1, 1, 0, s>>>(g, dtbits, dt_cur, dt_log, step, flags, t_end);
}
static int copy_blocks(long long n) {
  const long long b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}
void launch_pad(const Grid& gp, const Grid& gi, const double* U, double* Up, cudaStream_t s) {
  k_pad_copy<<<copy_blocks(8 * gi.N), 256, 0, s>>>(gp, gi, Up, const_cast<double*>(U), 0);
}
void launch_unpad(const Grid& gp, const Grid& gi, const double* Up, double* U, cudaStream_t s) {
  k_pad_copy<<<copy_blocks(8 * gi.N), 256, 0, s>>>(gp, gi, const_cast<double*>(Up), U, 1);
}
void launch_gather_sub(const Grid& gp, const Grid& gg, const int off[3], const double* Ug, double* Up,
                       cudaStream_t s) {
  k_gather_sub<<<copy_blocks(gp.N), 256, 0, s>>>(gp, gg, off[0], off[1], off[2], Ug, Up);
}
void launch_scatter_sub(const Grid& gp, const Grid& gg, const int off[3], const double* Up, double* Ug,
                        cudaStream_t s) {
  const long long M = (long long)(gp.hi[0] - gp.lo[0]) * (gp.hi[1] - gp.lo[1]) * (gp.hi[2] - gp.lo[2]);
  k_scatter_sub<<<copy_blocks(8 * M), 256, 0, s>>>(gp, gg, off[0], off[1], off[2], Up, Ug);
}
void launch_fill_ghosts(const Grid& gp, double* Up, cudaStream_t s) {
  k_fill_ghosts<<<copy_blocks(gp.N), 256, 0, s>>>(gp, Up);
}
void launch_diagnostics(const Grid& g, const double* U, double* red, int nb, cudaStream_t s) {
  // partials live after the 9 final values
  k_diag_partial<<<nb, DIAG_T, 0, s>>>(g, U, red + 9, nb);
  k_diag_final<<<1, DIAG_T, 0, s>>>(red + 9, red, nb);
}
}  // namespace mhd
