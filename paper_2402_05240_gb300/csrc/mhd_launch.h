// mhd_launch.h -- host-side declarations of the kernel launchers (internal).
#pragma once

#include <cuda_runtime.h>

namespace mhd {

struct df;  // double-float number (mhd_df.cuh)

// thread block of the per-cell kernels: BX x BY cells of one z plane
constexpr int BX = 32, BY = 4;
inline long long cell_blocks(int nx, int ny, int nz) {
  return (long long)((nx + BX - 1) / BX) * ((ny + BY - 1) / BY) * nz;
}

struct Grid {
  int n[3];          // nx, ny, nz
  long long N;       // nx * ny * nz
  double d[3];       // dx, dy, dz
  double id[3];      // 1/dx, 1/dy, 1/dz
  double gamma;
  double gm1, igm1;  // gamma - 1 and 1/(gamma - 1)
  double rho_floor, p_floor;
  double cfl;
  // interior box [lo, hi) of a padded grid (outflow boundaries): the CFL
  // reduction and the floor counters cover it only; lo = 0, hi = n otherwise
  int lo[3], hi[3];
  int bc[3];         // boundary condition per axis of the caller's grid (0 periodic, 1 outflow)
};

// A field-major array as a table of field pointers (a kernel parameter):
// field q of cell c is f[q][c].
template <class T, int K> struct Fields {
  T* f[K];
};

// the K field pointers of a field-major array with N cells per field (all
// null for a null base)
template <int K, class T> __host__ __device__ inline Fields<T, K> fields(T* base, long long N) {
  Fields<T, K> r;
#pragma unroll
  for (int q = 0; q < K; ++q) r.f[q] = base ? base + q * N : nullptr;
  return r;
}

// Intermediates of the three-pass PPMC reverse (per cell: the cotangents of
// the two limited interface deviations, 7 + 7, of the eigensystem fields,
// 17, and of the cell's own state after the back-projection, 7).
constexpr int kPpmcRevFields = 38;

// Launchers of the step kernels for compute type T (double: FP64 step,
// float: FP32-bulk step); all asynchronous on stream s.
template <class T> struct Launch {
  // Er (may be null): also the cells' reference fields -(v x B_cc), 3 x N
  static void prim(const Grid& g, double* U, T* W, unsigned long long* dtbits, unsigned* flags,
                   unsigned long long* floors, cudaStream_t s, T* Er = nullptr);
  static void flux_pcm(const Grid& g, int a, const T* W, const double* U, T* F, cudaStream_t s);  // axis a
  static void recon(const Grid& g, int rc, int a, const T* W, T* WL, T* WR, cudaStream_t s);
  static void flux_hlld(const Grid& g, int a, const T* WL, const T* WR, const T* Bf, T* F, cudaStream_t s);
  // Er: the reference fields written with W (null: formed from W)
  static void emf(const Grid& g, const T* W, const T* F, T* E, cudaStream_t s, const T* Er = nullptr);
  static void update_half(const Grid& g, const double* U, const T* F, const T* E, const double* dtp, T* W, T* Bh,
                          unsigned* flags, cudaStream_t s, T* Er = nullptr);
  static void update_full(const Grid& g, double* U, const T* F, const T* E, const double* dtp, cudaStream_t s);
  static void widen(const T* src, double* dst, long long n, cudaStream_t s);
  static void narrow(const double* src, T* dst, long long n, cudaStream_t s);
};

// Launchers of the adjoint (reverse-sweep) kernels for compute type T.
template <class T> struct AdjLaunch {
  static void floors(const Grid& g, const double* U, const T* F, const T* E, double dt, const double* gUp, double* gU,
                     T* gBccF, cudaStream_t s);
  // part != nullptr: also the block partials of the step-size cotangent
  // (fluxes Fs and edge fields Es of the update being reversed)
  static void update(const Grid& g, int mode, double h, const double* g5src, const double* gUpF, const T* gBcc,
                     const T* gBfx, double* gU, T* gF, T* gE, cudaStream_t s, const T* Fs = nullptr,
                     const T* Es = nullptr, double* part = nullptr);
  // reverse of dt = C_CFL / r_max: argmax cell of the rate, g_dt from the
  // partials of both update reverses (nparts per mode), g_dt d dt/dU into gU;
  // out = {g_dt, dt, cell}
  static void cfl_term(const Grid& g, const double* U, const T* W, const unsigned long long* rbits, const double* part,
                       long long nparts, unsigned long long* idx, double* gU, double* out, cudaStream_t s);
  static void emf(const Grid& g, const T* W, const T* F, const T* gE, T* gF, T* gW, cudaStream_t s);
  static void hlld(const Grid& g, int a, bool pcm, const T* WL, const T* WR, const T* Wn, const double* U, const T* Bh,
                   const T* gF, T* gWL, T* gWR, T* gBf, cudaStream_t s);
  static void pcm_gather(const Grid& g, int a, const T* gWL, const T* gWR, T* gW, cudaStream_t s);
  template <int R>
  static void recon_r(const Grid& g, int a, const T* W, const T* gWL, const T* gWR, T* S, T* gW, cudaStream_t s);
  // X: scratch of the PPMC reverse (kPpmcRevFields arrays of N values; unused
  // for the other reconstructions)
  static void recon(const Grid& g, int rc, int a, const T* W, const T* gWL, const T* gWR, T* S, T* gW,
                    const Fields<T, kPpmcRevFields>& X, cudaStream_t s);
  static void prim(const Grid& g, bool half, const double* U, const double* Uh, const T* Bh, const T* gW, double* g5,
                   T* gBcc, cudaStream_t s);
  static void faces_n(const Grid& g, const double* g5, const T* gBcc, const T* gBf, double* gU, cudaStream_t s);
  static void fwd_half_keep(const Grid& g, const double* U, const T* F, const T* E, double dt, T* W, T* Bh, double* Uh,
                            cudaStream_t s);
  static void hlld_batch(int n, double gamma, const double* wl, const double* wr, const double* bn, const double* gf,
                         double* gwl, double* gwr, double* gbn, double* f, cudaStream_t s);
};

// Scalars of the current step on the device, written with its dt by
// k_set_dt / k_finish_dt so that the update kernels read the dt-derived
// factors instead of forming them per cell.  Lives in the context's scalar
// area (kStepScalarDoubles doubles).
struct StepScalars {
  double dt, t;           // step size, simulated time of the current run
  double h_half;          // dt / 2 (Step 5)
  double hd_full[3];      // dt / d_a (Step 9)
  double hd_half[3];      // (dt / 2) / d_a (Step 5)
  float hd_half_f[3];     // hd_half rounded to float (FP32-bulk half step)
  float hd_full_hi[3];    // hd_full and hd_half as float pairs (the
  float hd_full_lo[3];    // double-float conversion of the double values)
  float hd_half_hi[3];
  float hd_half_lo[3];
};
constexpr int kStepScalarDoubles = 32;
static_assert(sizeof(StepScalars) <= kStepScalarDoubles * sizeof(double), "step scalars fit their area");

// dt of a step given by the caller
void launch_set_dt(const Grid& g, double* dt_cur, double value, cudaStream_t s);
// dt of the next step from the reduction word (C_CFL = g.cfl); t_end = +inf
// for no end time
void launch_finish_dt(const Grid& g, unsigned long long* dtbits, double* dt_cur, double* dt_log, int step,
                      unsigned* flags, double t_end, cudaStream_t s);

// Diagnostics scratch layout (doubles): the 9 results (8 field sums, then
// max |div B|), then per partial block 9 partials (field-major: red[9 + f nb
// + b]), then per block the 8 compensation terms of the field sums
// (red[9 + (9 + f) nb + b]).  One partial block reduces kDiagCells cells.
constexpr long long kDiagCells = 1024;
constexpr long long diag_blocks(long long N) { return N < 1 ? 1 : (N + kDiagCells - 1) / kDiagCells; }
constexpr long long diag_scratch_doubles(long long nb) { return 9 + 17 * nb; }

// max |div B| and field sums of a state into red[0..8]; red holds
// diag_scratch_doubles(nb) doubles, nb = diag_blocks(g.N)
void launch_diagnostics(const Grid& g, const double* U, double* red, int nb, cudaStream_t s);

// outflow boundaries: copy the caller's state U (grid gi) into the interior
// box of the padded state Up (grid gp), copy it back, and fill every ghost
// cell of Up (outside gp's interior box) from the nearest interior cell
void launch_pad(const Grid& gp, const Grid& gi, const double* U, double* Up, cudaStream_t s);
void launch_unpad(const Grid& gp, const Grid& gi, const double* Up, double* U, cudaStream_t s);
void launch_fill_ghosts(const Grid& gp, double* Up, cudaStream_t s);
// subdomains: gather the padded subdomain state (interior + halo, periodic
// wrap of the global grid gg) at global offset off; scatter its interior back
void launch_gather_sub(const Grid& gp, const Grid& gg, const int off[3], const double* Ug, double* Up,
                       cudaStream_t s);
void launch_scatter_sub(const Grid& gp, const Grid& gg, const int off[3], const double* Up, double* Ug,
                        cudaStream_t s);

}  // namespace mhd
