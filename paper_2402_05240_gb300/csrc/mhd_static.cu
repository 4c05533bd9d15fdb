// mhd_static.cu -- mhd_diagnostics_static: the diagnostics reduction without
// any device allocation (no context, no cudaMalloc / cudaFree).
//
// Some callers cannot allocate device memory when they need a diagnostic:
// a host whose whole device memory was handed to another allocator up front
// (a framework's caching pool, an MPI library's registered buffers), where an
// extra cudaMalloc fails; or a tight step loop where cudaMalloc/cudaFree
// would add implicit device synchronisation.  This entry point serves them:
// the per-block partial sums live in a file-scope device array that every GPU
// loading the library holds from load time until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mhd_api.h"
#include "mhd_launch.h"

namespace {

// Largest grid served: 512^3 cells -> 131072 partial blocks.
constexpr long long kMaxCells = 134217728LL;
constexpr long long kMaxBlocks = mhd::diag_blocks(kMaxCells);
// The layout the diagnostics kernels write (mhd_launch.h): 9 results, then 9
// partials and 8 compensation terms per block -- 9 + 17 * 131072 doubles,
// 17.8 MB.
constexpr long long kScratchDoubles = mhd::diag_scratch_doubles(kMaxBlocks);
static_assert(kScratchDoubles == 9 + 17 * 131072LL, "static scratch sized for 512^3 cells");

__device__ __align__(256) double g_diag_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

// Device address of the static scratch on the current device.  In host code
// the array's name is only a host-side handle, so the address is looked up
// once per device with cudaGetSymbolAddress while that device is current.
int scratch_on_current_device(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return MHD_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return MHD_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_diag_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MHD_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[dev];
  return MHD_OK;
}

}  // namespace

extern "C" int mhd_diagnostics_static(const mhd_config* cfg, const double* U_dev, void* stream,
                                      double* divb_max_host, double totals_host[8]) {
  if (!cfg || !U_dev || !divb_max_host || !totals_host) return MHD_ERR_ARG;
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return MHD_ERR_ARG;
  if (!(cfg->dx > 0) || !(cfg->dy > 0) || !(cfg->dz > 0)) return MHD_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (cfg->bc[a] != MHD_BC_PERIODIC && cfg->bc[a] != MHD_BC_OUTFLOW && cfg->bc[a] != MHD_BC_HALO) return MHD_ERR_ARG;
  const long long N = (long long)cfg->nx * cfg->ny * cfg->nz;
  if (N > kMaxCells || cfg->nz > 65535) return MHD_ERR_TOO_LARGE;
  double* scratch = nullptr;
  int st = scratch_on_current_device(&scratch);
  if (st != MHD_OK) return st;
  mhd::Grid g;
  g.n[0] = cfg->nx;
  g.n[1] = cfg->ny;
  g.n[2] = cfg->nz;
  g.N = N;
  g.d[0] = cfg->dx;
  g.d[1] = cfg->dy;
  g.d[2] = cfg->dz;
  for (int a = 0; a < 3; ++a) g.id[a] = 1.0 / g.d[a];
  g.gm1 = cfg->gamma - 1.0;
  g.igm1 = cfg->gamma > 1.0 ? 1.0 / (cfg->gamma - 1.0) : 0.0;
  g.gamma = cfg->gamma;
  g.rho_floor = cfg->rho_floor;
  g.p_floor = cfg->p_floor;
  g.cfl = cfg->cfl;
  for (int a = 0; a < 3; ++a) {
    g.lo[a] = 0;
    g.hi[a] = g.n[a];
    g.bc[a] = cfg->bc[a];
  }
  const long long nblk = mhd::diag_blocks(N);
  // the size check above bounds nblk; this one ties the launch to the array
  if (mhd::diag_scratch_doubles(nblk) > kScratchDoubles) return MHD_ERR_TOO_LARGE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // Every partial the final pass reads is written by the partial pass of this
  // call, so nothing in the scratch has to start at zero.
  mhd::launch_diagnostics(g, U_dev, scratch, (int)nblk, s);
  if (cudaGetLastError() != cudaSuccess) return MHD_ERR_CUDA;
  double out[9];
  if (cudaMemcpyAsync(out, scratch, sizeof(out), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ERR_CUDA;
  *divb_max_host = out[8];
  for (int f = 0; f < 8; ++f) totals_host[f] = out[f];
  return MHD_OK;
}
