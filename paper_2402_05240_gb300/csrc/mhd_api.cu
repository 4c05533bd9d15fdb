// mhd_api.cu -- the C ABI (include/mhd_api.h): context, workspace, step
// sequencing.  Every numerical stage runs in the kernels of mhd_kernels.cuh.
#include <cuda_runtime.h>

#include <sys/mman.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mhd_api.h"
#include "mhd_df.cuh"
#include "mhd_launch.h"

using mhd::Grid;
using mhd::Launch;

struct ProfRec {
  int stage;
  cudaEvent_t a, b;
};

struct mhd_ctx {
  mhd_config cfg;
  Grid g;               // grid of the step kernels (padded along outflow axes)
  Grid gi;              // the caller's grid
  double* Up;           // padded state (outflow boundaries), else nullptr
  cudaStream_t stream;
  size_t ts;            // bytes of the compute type
  void* ws;             // one workspace allocation
  size_t ws_bytes;
  // typed views into ws (element type = compute type)
  void *W, *F, *E, *WL, *WR, *Bh;
  void* Er;                     // cell reference fields -(v x B_cc) written with W (step path)
  double* scal;                 // mhd::StepScalars of the current step ([0] dt, [1] t)
  unsigned long long* dtbits;   // [0] dt reduction word
  unsigned long long* floors;   // [0..1] floor counters
  unsigned* flags;              // [0] error flags
  double* red;                  // diagnostics partials
  double* host_state;           // lazily allocated device copy for mhd_run_host
  size_t red_count;
  void* adj_ws;                 // adjoint workspace, allocated by the first adjoint call
  size_t adj_bytes;
  // optional per-stage CUDA-event timing (mhd_profile_enable)
  int prof_on;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used;
};

namespace {

// compute type of each precision mode
template <class T> struct Tag { using type = T; };
template <class Fn> int with_type(int precision, Fn&& fn) {
  if (precision == MHD_FP32_BULK) return fn(Tag<float>{});
  if (precision == MHD_FP64_DF) return fn(Tag<mhd::df>{});
  return fn(Tag<double>{});
}
template <class Fn> int with_adj_type(int precision, Fn&& fn) { return with_type(precision, fn); }
#define MHD_T typename decltype(t)::type

constexpr size_t kAlign = 256;
size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t W, F, E, WL, WR, Bh, Er, scal, dtbits, floors, flags, red, Up, total;
};

bool padded(const mhd_config& c) {
  return c.bc[0] != MHD_BC_PERIODIC || c.bc[1] != MHD_BC_PERIODIC || c.bc[2] != MHD_BC_PERIODIC;
}
bool has_halo(const mhd_config& c) {
  return c.bc[0] == MHD_BC_HALO || c.bc[1] == MHD_BC_HALO || c.bc[2] == MHD_BC_HALO;
}

// cells per axis of the step kernels' grid: MHD_GHOST more on each side of
// an outflow axis
void padded_dims(const mhd_config& c, int n[3], int lo[3]) {
  const int ni[3] = {c.nx, c.ny, c.nz};
  for (int a = 0; a < 3; ++a) {
    lo[a] = c.bc[a] != MHD_BC_PERIODIC ? MHD_GHOST : 0;
    n[a] = ni[a] + 2 * lo[a];
  }
}

size_t red_blocks(long long N) { return (size_t)mhd::diag_blocks(N); }

Layout layout_of(const mhd_config& c) {
  int np[3], lo[3];
  padded_dims(c, np, lo);
  const size_t N = (size_t)np[0] * np[1] * np[2];
  const size_t Ni = (size_t)c.nx * c.ny * c.nz;
  const size_t ts = c.precision == MHD_FP32_BULK ? 4 : 8;
  Layout L;
  size_t off = 0;
  L.W = off;
  off += up(8 * N * ts);
  L.F = off;
  off += up(21 * N * ts);
  L.E = off;
  off += up(3 * N * ts);
  L.WL = off;
  off += up(7 * N * ts);
  L.WR = off;
  off += up(7 * N * ts);
  L.Bh = off;
  off += up(3 * N * ts);
  L.Er = off;
  off += up(3 * N * ts);
  L.scal = off;
  off += up(mhd::kStepScalarDoubles * sizeof(double));
  L.dtbits = off;
  off += up(sizeof(unsigned long long));
  L.floors = off;
  off += up(2 * sizeof(unsigned long long));
  L.flags = off;
  off += up(sizeof(unsigned));
  L.red = off;
  off += up((size_t)mhd::diag_scratch_doubles((long long)red_blocks((long long)Ni)) * sizeof(double));
  L.Up = off;
  if (padded(c)) off += up(8 * N * sizeof(double));
  L.total = off;
  return L;
}

int check_cfg(const mhd_config* c) {
  if (!c) return MHD_ERR_ARG;
  if (c->nx < 4 || c->ny < 4 || c->nz < 4) return MHD_ERR_ARG;
  if ((long long)c->nx * c->ny > (1ll << 31) || c->nz > 65535) return MHD_ERR_ARG;
  if (!(c->dx > 0) || !(c->dy > 0) || !(c->dz > 0)) return MHD_ERR_ARG;
  if (!(c->gamma > 1.0) || !std::isfinite(c->gamma)) return MHD_ERR_ARG;
  if (!(c->cfl > 0.0) || c->cfl > 1.0) return MHD_ERR_ARG;
  if (c->recon < MHD_RECON_PCM || c->recon > MHD_RECON_PLM_PRIM) return MHD_ERR_ARG;
  if (c->precision != MHD_FP64 && c->precision != MHD_FP32_BULK && c->precision != MHD_FP64_DF) return MHD_ERR_ARG;
  if (!(c->rho_floor > 0) || !(c->p_floor > 0)) return MHD_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (c->bc[a] != MHD_BC_PERIODIC && c->bc[a] != MHD_BC_OUTFLOW && c->bc[a] != MHD_BC_HALO) return MHD_ERR_ARG;
  if (has_halo(*c) && (c->bc[0] == MHD_BC_OUTFLOW || c->bc[1] == MHD_BC_OUTFLOW || c->bc[2] == MHD_BC_OUTFLOW))
    return MHD_ERR_ARG;  // subdomains of periodic global grids only
  int np[3], lo[3];
  padded_dims(*c, np, lo);
  if ((long long)np[0] * np[1] > (1ll << 31) || np[2] > 65535) return MHD_ERR_ARG;
  // the step kernels index cells with 32-bit integers
  if ((long long)np[0] * np[1] * np[2] > 2147483647LL) return MHD_ERR_ARG;
  return MHD_OK;
}

int cuda_status() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MHD_OK : MHD_ERR_CUDA;
}

template <class T> T* as(void* p) { return static_cast<T*>(p); }

cudaEvent_t next_event(mhd_ctx* c) {
  if (c->ev_used == c->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    c->ev_pool.push_back(e);
  }
  return c->ev_pool[c->ev_used++];
}

// Runs one launch; with profiling on, brackets it with events on the stream.
template <class Fn> void prof(mhd_ctx* c, int stage, Fn&& fn) {
  if (!c->prof_on) {
    fn();
    return;
  }
  ProfRec r;
  r.stage = stage;
  r.a = next_event(c);
  r.b = next_event(c);
  cudaEventRecord(r.a, c->stream);
  fn();
  cudaEventRecord(r.b, c->stream);
  c->prof.push_back(r);
}

// Steps 2-9 given W^n (in ctx->W) and dt in scal[0]; U in place.
template <class T> void step_body(mhd_ctx* c, double* U, int recon) {
  const Grid& g = c->g;
  cudaStream_t s = c->stream;
  T* W = as<T>(c->W);
  T* F = as<T>(c->F);
  T* E = as<T>(c->E);
  for (int a = 0; a < 3; ++a)  // Steps 2-3
    prof(c, MHD_STAGE_FLUX_PCM, [&] { Launch<T>::flux_pcm(g, a, W, U, F, s); });
  T* Er = as<T>(c->Er);
  prof(c, MHD_STAGE_EMF, [&] { Launch<T>::emf(g, W, F, E, s, Er); });        // Step 4
  prof(c, MHD_STAGE_UPDATE_HALF,
       [&] { Launch<T>::update_half(g, U, F, E, c->scal, W, as<T>(c->Bh), c->flags, s, Er); });  // Step 5
  for (int a = 0; a < 3; ++a) {                                               // Steps 6-7
    prof(c, MHD_STAGE_RECON, [&] { Launch<T>::recon(g, recon, a, W, as<T>(c->WL), as<T>(c->WR), s); });
    prof(c, MHD_STAGE_FLUX_HLLD,
         [&] { Launch<T>::flux_hlld(g, a, as<T>(c->WL), as<T>(c->WR), as<T>(c->Bh), F, s); });
  }
  prof(c, MHD_STAGE_EMF, [&] { Launch<T>::emf(g, W, F, E, s, Er); });        // Step 8
  prof(c, MHD_STAGE_UPDATE_FULL, [&] { Launch<T>::update_full(g, U, F, E, c->scal, s); });  // Step 9
}

constexpr double kNoEnd = HUGE_VAL;

// Outflow boundaries: the step kernels work on the padded copy Up of the
// caller's state, whose ghost cells are refilled from the interior after
// every step (before the primitives, floors and CFL maximum of the next).
double* enter(mhd_ctx* c, const double* U) {
  if (!c->Up) return const_cast<double*>(U);
  mhd::launch_pad(c->g, c->gi, U, c->Up, c->stream);
  mhd::launch_fill_ghosts(c->g, c->Up, c->stream);
  return c->Up;
}
void leave(mhd_ctx* c, double* U) {
  if (c->Up) mhd::launch_unpad(c->g, c->gi, c->Up, U, c->stream);
}
void refill(mhd_ctx* c, double* S) {
  if (c->Up) mhd::launch_fill_ghosts(c->g, S, c->stream);
}

// arm the reduction word (+0.0: the maximum of non-negative rates) and the
// run's simulated time, then W^0 and the CFL maximum of U^0
template <class T> void run_begin(mhd_ctx* c, double* U) {
  cudaStream_t s = c->stream;
  cudaMemsetAsync(c->dtbits, 0, sizeof(unsigned long long), s);
  cudaMemsetAsync(c->scal + 1, 0, sizeof(double), s);
  Launch<T>::prim(c->g, U, as<T>(c->W), c->dtbits, c->flags, nullptr, s, as<T>(c->Er));
}

// one device-dt step: dt (Step 1), Steps 2-9, then floors, W^{n+1} and the
// next CFL maximum
template <class T> void run_one(mhd_ctx* c, double* U, double* dt_log, int n, double t_end) {
  const Grid& g = c->g;
  cudaStream_t s = c->stream;
  prof(c, MHD_STAGE_DT, [&] { mhd::launch_finish_dt(g, c->dtbits, c->scal, dt_log, n, c->flags, t_end, s); });
  step_body<T>(c, U, c->cfg.recon);
  refill(c, U);
  prof(c, MHD_STAGE_PRIM,
       [&] { Launch<T>::prim(g, U, as<T>(c->W), c->dtbits, c->flags, c->floors, s, as<T>(c->Er)); });
}

template <class T> int run_steps(mhd_ctx* c, double* U, int nsteps, double* dt_log) {
  double* S = enter(c, U);
  run_begin<T>(c, S);
  for (int n = 0; n < nsteps; ++n) run_one<T>(c, S, dt_log, n, kNoEnd);
  leave(c, U);
  return cuda_status();
}

// steps until the simulated time reaches t_end (the last step shortened);
// reads the time back after every step
template <class T> int evolve_to(mhd_ctx* c, double* U, double t_end, int max_steps, double* t_out, int* n_out) {
  cudaStream_t s = c->stream;
  double* S = enter(c, U);
  run_begin<T>(c, S);
  double t = 0.0;
  int n = 0, st = MHD_OK;
  while (st == MHD_OK && n < max_steps && t < t_end) {
    run_one<T>(c, S, nullptr, n, t_end);
    ++n;
    unsigned fl = 0;
    if (cudaMemcpyAsync(&t, c->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&fl, c->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return MHD_ERR_CUDA;
    if (fl & 1u) st = MHD_ERR_NONFINITE;
    else if (fl & 2u) st = MHD_ERR_DT;
  }
  leave(c, U);
  if (t_out) *t_out = t;
  if (n_out) *n_out = n;
  if (st != MHD_OK) return st;
  return cuda_status();
}

template <class T> int one_step(mhd_ctx* c, double* U, double dt, double* next_dt) {
  const Grid& g = c->g;
  cudaStream_t s = c->stream;
  mhd::launch_set_dt(c->g, c->scal, dt, s);
  double* S = enter(c, U);
  Launch<T>::prim(g, S, as<T>(c->W), nullptr, c->flags, nullptr, s, as<T>(c->Er));
  step_body<T>(c, S, c->cfg.recon);
  refill(c, S);
  if (next_dt) cudaMemsetAsync(c->dtbits, 0, sizeof(unsigned long long), s);
  Launch<T>::prim(g, S, as<T>(c->W), next_dt ? c->dtbits : nullptr, c->flags, c->floors, s);
  leave(c, U);
  if (!next_dt) return cuda_status();
  mhd::launch_finish_dt(g, c->dtbits, c->scal, nullptr, 0, c->flags, kNoEnd, s);
  double v = 0;
  if (cudaMemcpyAsync(&v, c->scal, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ERR_CUDA;
  *next_dt = v;
  if (!(v > 0.0) || !std::isfinite(v)) return MHD_ERR_DT;
  return MHD_OK;
}

template <class T> int step_sub(mhd_ctx* c, const double* Ug, const int gn[3], const int off[3], double dt,
                                double* Ug_out) {
  const Grid& g = c->g;
  cudaStream_t s = c->stream;
  Grid gg = c->gi;
  for (int a = 0; a < 3; ++a) gg.n[a] = gn[a];
  gg.N = (long long)gn[0] * gn[1] * gn[2];
  mhd::launch_set_dt(c->g, c->scal, dt, s);
  mhd::launch_gather_sub(g, gg, off, Ug, c->Up, s);
  Launch<T>::prim(g, c->Up, as<T>(c->W), nullptr, c->flags, nullptr, s, as<T>(c->Er));
  step_body<T>(c, c->Up, c->cfg.recon);
  Launch<T>::prim(g, c->Up, as<T>(c->W), nullptr, c->flags, c->floors, s);
  mhd::launch_scatter_sub(g, gg, off, c->Up, Ug_out, s);
  return cuda_status();
}

template <class T> int dt_sub(mhd_ctx* c, const double* Ug, const int gn[3], const int off[3], double* dt_host) {
  cudaStream_t s = c->stream;
  Grid gg = c->gi;
  for (int a = 0; a < 3; ++a) gg.n[a] = gn[a];
  gg.N = (long long)gn[0] * gn[1] * gn[2];
  mhd::launch_gather_sub(c->g, gg, off, Ug, c->Up, s);
  cudaMemsetAsync(c->dtbits, 0, sizeof(unsigned long long), s);
  Launch<T>::prim(c->g, c->Up, as<T>(c->W), c->dtbits, c->flags, nullptr, s);
  mhd::launch_finish_dt(c->g, c->dtbits, c->scal, nullptr, 0, c->flags, kNoEnd, s);
  double v = 0;
  if (cudaMemcpyAsync(&v, c->scal, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ERR_CUDA;
  *dt_host = v;
  if (!(v > 0.0) || !std::isfinite(v)) return MHD_ERR_DT;
  return MHD_OK;
}

// sizes and offset of a subdomain inside the state handed to mhd_step_sub / mhd_dt_sub
int check_sub(mhd_ctx* c, const int gn[3], const int off[3]) {
  for (int a = 0; a < 3; ++a) {
    if (gn[a] < c->gi.n[a] || off[a] < 0 || off[a] + c->gi.n[a] > gn[a]) return MHD_ERR_ARG;
    if (c->cfg.bc[a] == MHD_BC_PERIODIC && gn[a] != c->gi.n[a]) return MHD_ERR_ARG;
  }
  if ((long long)gn[0] * gn[1] > (1ll << 31) || gn[2] > 65535) return MHD_ERR_ARG;
  return MHD_OK;
}

// ---- adjoint ----------------------------------------------------------------
// Adjoint buffers (compute type T): forward intermediates W^n[8], F^n[21],
// W^{n+1/2}[8], B^{n+1/2}[3], W_L/W_R of the three axes [21+21], F^{n+1/2}[21],
// E[3]; cotangents gF[21], gE[3], gW[8], gWL[7], gWR[7], recon slots[36],
// gBf[3], gBcc[3], gBccF[3]; in double the half-step hydro state[5] and g5[5];
// then the per-block partials of the dt cotangent (two per block) and a few
// scalars for the reverse of the CFL dt.  W^n, F^n, E, B^{n+1/2}, gWL and
// gWR live in the context's step workspace (W, F, E, Bh, WL, WR, 49 words),
// which holds nothing between calls (every step entry point recomputes W
// first); the adjoint allocates the other 148 words and the doubles.
constexpr size_t kAdjOwnWords = 197 - 49;
size_t adj_part_count(const mhd_config& c) { return (size_t)mhd::cell_blocks(c.nx, c.ny, c.nz); }
size_t adj_bytes_of(const mhd_config& c) {
  const size_t N = (size_t)c.nx * c.ny * c.nz;
  const size_t ts = c.precision == MHD_FP32_BULK ? 4 : 8;
  return up(kAdjOwnWords * N * ts) + up(10 * N * sizeof(double)) +
         up((2 * adj_part_count(c) + 8) * sizeof(double)) + 4 * kAlign;
}

template <class T> struct AdjView {
  T *Wn, *Fn, *Wh, *Bh, *WLa, *WRa, *Fh, *Eh, *gF, *gE, *gW, *gWL, *gWR, *gS, *gBf, *gBcc, *gBccF;
  double *Uh, *g5;
  double* part;              // [2][nparts] dt-cotangent partials of the Step 9 and Step 5 reverses
  long long nparts;
  double* out;               // [3] g_dt, dt, maximising cell
  unsigned long long* idx;   // argmax word
};

// Scratch of the three-pass PPMC reverse of axis a: arrays that are dead
// while it runs -- the corrector fluxes F^{n+1/2} (used by the Step 9 and
// Step 8 reverses, which come first), the interface states of axis a and the
// flux cotangents of axis a (both used up by that axis's HLLD reverse, which
// comes just before).
template <class T> mhd::Fields<T, mhd::kPpmcRevFields> ppmc_rev_scratch(const AdjView<T>& b, int a, long long N) {
  mhd::Fields<T, mhd::kPpmcRevFields> X;
  int q = 0;
  for (int f = 0; f < 21; ++f) X.f[q++] = b.Fh + f * N;
  for (int f = 0; f < 7; ++f) X.f[q++] = b.WLa + (a * 7 + f) * N;
  for (int f = 0; f < 7; ++f) X.f[q++] = b.WRa + (a * 7 + f) * N;
  for (int f = 0; f < 3; ++f) X.f[q++] = b.gF + (a * 7 + f) * N;
  return X;
}

template <class T> int adj_view(mhd_ctx* c, AdjView<T>& v) {
  if (!c->adj_ws) {
    const size_t b = adj_bytes_of(c->cfg);
    cudaGetLastError();
    if (cudaMalloc(&c->adj_ws, b) != cudaSuccess) {
      cudaGetLastError();
      c->adj_ws = nullptr;
      return MHD_ERR_OOM;
    }
    c->adj_bytes = b;
  }
  const size_t N = (size_t)c->g.N;
  T* p = static_cast<T*>(c->adj_ws);
  auto take = [&](size_t n) {
    T* q = p;
    p += n * N;
    return q;
  };
  v.Wn = as<T>(c->W);
  v.Fn = as<T>(c->F);
  v.Eh = as<T>(c->E);
  v.Bh = as<T>(c->Bh);
  v.gWL = as<T>(c->WL);
  v.gWR = as<T>(c->WR);
  v.Wh = take(8);
  v.WLa = take(21);
  v.WRa = take(21);
  v.Fh = take(21);
  v.gF = take(21);
  v.gE = take(3);
  v.gW = take(8);
  v.gS = take(36);
  v.gBf = take(3);
  v.gBcc = take(3);
  v.gBccF = take(3);
  static_assert(8 + 21 * 4 + 3 + 8 + 36 + 3 * 3 == kAdjOwnWords, "adjoint buffers");
  char* d = reinterpret_cast<char*>(c->adj_ws) + up(kAdjOwnWords * N * sizeof(T));
  v.Uh = reinterpret_cast<double*>(d);
  v.g5 = v.Uh + 5 * N;
  v.nparts = (long long)adj_part_count(c->cfg);
  v.part = reinterpret_cast<double*>(d + up(10 * N * sizeof(double)));
  v.out = v.part + 2 * v.nparts;
  v.idx = reinterpret_cast<unsigned long long*>(v.out + 4);
  return MHD_OK;
}

// cfl: dt is the CFL dt of U^n (Step 1) and its reverse is added: the
// update reverses also produce the dt cotangent, and cfl_term adds
// g_dt d dt/dU^n.  dt_host/gdt_host (may be null) receive dt and g_dt.
template <class T>
int adjoint_step(mhd_ctx* c, const double* Un, double dt, const double* gUp, double* gU, bool cfl = false,
                 double* dt_host = nullptr, double* gdt_host = nullptr) {
  AdjView<T> b;
  int st = adj_view<T>(c, b);
  if (st != MHD_OK) return st;
  const Grid& g = c->g;
  cudaStream_t s = c->stream;
  const long long N = g.N;
  double* U = const_cast<double*>(Un);  // read only: k_prim writes U only with floors on
  const int rc = c->cfg.recon;
  if (cfl) {
    // Step 1's reduction, read back for the host-side dt of the recompute
    cudaMemsetAsync(c->dtbits, 0, sizeof(unsigned long long), s);
    Launch<T>::prim(g, U, b.Wn, c->dtbits, c->flags, nullptr, s);
    unsigned long long bits = 0;
    unsigned fl = 0;
    if (cudaMemcpyAsync(&bits, c->dtbits, sizeof(bits), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
    if (cudaMemcpyAsync(&fl, c->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ERR_CUDA;
    if (fl & 1u) return MHD_ERR_NONFINITE;
    double r;
    std::memcpy(&r, &bits, sizeof(r));
    dt = g.cfl / r;
    if (!(dt > 0.0) || !std::isfinite(dt)) return MHD_ERR_DT;
  }
  double* part0 = cfl ? b.part : nullptr;
  double* part1 = cfl ? b.part + b.nparts : nullptr;
  // forward recompute (Steps 1-8; W^n is already in place after the dt reduction)
  if (!cfl) Launch<T>::prim(g, U, b.Wn, nullptr, c->flags, nullptr, s);
  for (int a = 0; a < 3; ++a) Launch<T>::flux_pcm(g, a, b.Wn, U, b.Fn, s);
  Launch<T>::emf(g, b.Wn, b.Fn, b.Eh, s);
  mhd::AdjLaunch<T>::fwd_half_keep(g, U, b.Fn, b.Eh, dt, b.Wh, b.Bh, b.Uh, s);
  for (int a = 0; a < 3; ++a) {
    Launch<T>::recon(g, rc, a, b.Wh, b.WLa + a * 7 * N, b.WRa + a * 7 * N, s);
    Launch<T>::flux_hlld(g, a, b.WLa + a * 7 * N, b.WRa + a * 7 * N, b.Bh, b.Fh, s);
  }
  Launch<T>::emf(g, b.Wh, b.Fh, b.Eh, s);
  // reverse: Step 9 (floors, full update)
  mhd::AdjLaunch<T>::floors(g, U, b.Fh, b.Eh, dt, gUp, gU, b.gBccF, s);
  mhd::AdjLaunch<T>::update(g, 0, dt, gU, gUp + 5 * N, b.gBccF, nullptr, gU, b.gF, b.gE, s, b.Fh, b.Eh, part0);
  // Step 8 (edge fields, half-step reference fields)
  mhd::AdjLaunch<T>::emf(g, b.Wh, b.Fh, b.gE, b.gF, b.gW, s);
  // Steps 7-6 per axis (HLLD, reconstruction)
  for (int a = 0; a < 3; ++a) {
    mhd::AdjLaunch<T>::hlld(g, a, false, b.WLa + a * 7 * N, b.WRa + a * 7 * N, nullptr, nullptr, b.Bh, b.gF, b.gWL,
                            b.gWR, b.gBf, s);
    mhd::AdjLaunch<T>::recon(g, rc, a, b.Wh, b.gWL, b.gWR, b.gS, b.gW, ppmc_rev_scratch<T>(b, a, N), s);
  }
  // Step 5 (primitives of the half state, half update)
  mhd::AdjLaunch<T>::prim(g, true, U, b.Uh, b.Bh, b.gW, b.g5, b.gBcc, s);
  // (the predictor edge fields, overwritten by Step 8's, again for the dt cotangent)
  if (cfl) Launch<T>::emf(g, b.Wn, b.Fn, b.Eh, s);
  mhd::AdjLaunch<T>::update(g, 1, 0.5 * dt, b.g5, nullptr, b.gBcc, b.gBf, gU, b.gF, b.gE, s, b.Fn, b.Eh, part1);
  // Step 4 (edge fields, reference fields of W^n)
  mhd::AdjLaunch<T>::emf(g, b.Wn, b.Fn, b.gE, b.gF, b.gW, s);
  // Steps 3-2 (HLLD on PCM states)
  for (int a = 0; a < 3; ++a) {
    mhd::AdjLaunch<T>::hlld(g, a, true, nullptr, nullptr, b.Wn, U, nullptr, b.gF, b.gWL, b.gWR, b.gBf, s);
    mhd::AdjLaunch<T>::pcm_gather(g, a, b.gWL, b.gWR, b.gW, s);
  }
  // Step 1 (primitives of U^n) and the face cotangents
  mhd::AdjLaunch<T>::prim(g, false, U, nullptr, nullptr, b.gW, b.g5, b.gBcc, s);
  mhd::AdjLaunch<T>::faces_n(g, b.g5, b.gBcc, b.gBf, gU, s);
  if (!cfl) return cuda_status();
  mhd::AdjLaunch<T>::cfl_term(g, U, b.Wn, c->dtbits, b.part, b.nparts, b.idx, gU, b.out, s);
  double o[3] = {0, 0, 0};
  if (cudaMemcpyAsync(o, b.out, sizeof(o), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ERR_CUDA;
  if (dt_host) *dt_host = o[1];
  if (gdt_host) *gdt_host = o[0];
  if (!(o[2] >= 0.0)) return MHD_ERR_DT;  // no cell reached the maximum
  return cuda_status();
}

template <class T>
int stage_recon_vjp(mhd_ctx* c, const double* U, int axis, int recon, const double* gWL, const double* gWR, double* gU) {
  AdjView<T> b;
  int st = adj_view<T>(c, b);
  if (st != MHD_OK) return st;
  const Grid& g = c->g;
  cudaStream_t s = c->stream;
  const long long N = g.N;
  Launch<T>::prim(g, const_cast<double*>(U), b.Wn, nullptr, c->flags, nullptr, s);
  Launch<T>::narrow(gWL, b.gWL, 7 * N, s);
  Launch<T>::narrow(gWR, b.gWR, 7 * N, s);
  cudaMemsetAsync(b.gW, 0, 8 * N * sizeof(T), s);
  cudaMemsetAsync(b.gBf, 0, 3 * N * sizeof(T), s);
  cudaMemsetAsync(gU, 0, 8 * N * sizeof(double), s);
  mhd::AdjLaunch<T>::recon(g, recon, axis, b.Wn, b.gWL, b.gWR, b.gS, b.gW, ppmc_rev_scratch<T>(b, axis, N), s);
  mhd::AdjLaunch<T>::prim(g, false, U, nullptr, nullptr, b.gW, b.g5, b.gBcc, s);
  mhd::AdjLaunch<T>::faces_n(g, b.g5, b.gBcc, b.gBf, gU, s);
  return cuda_status();
}

// ---- stage entry points ---------------------------------------------------
template <class T> int stage_prims(mhd_ctx* c, const double* U, double* Wout) {
  Launch<T>::prim(c->g, const_cast<double*>(U), as<T>(c->W), nullptr, c->flags, nullptr, c->stream);
  Launch<T>::widen(as<T>(c->W), Wout, 8 * c->g.N, c->stream);
  return cuda_status();
}

template <class T> int stage_fluxes(mhd_ctx* c, const double* U, int recon, double* Fout) {
  const Grid& g = c->g;
  cudaStream_t s = c->stream;
  Launch<T>::prim(g, const_cast<double*>(U), as<T>(c->W), nullptr, c->flags, nullptr, s);
  if (recon == MHD_RECON_PCM) {
    for (int a = 0; a < 3; ++a) Launch<T>::flux_pcm(g, a, as<T>(c->W), U, as<T>(c->F), s);
  } else {
    Launch<T>::narrow(U + 5 * g.N, as<T>(c->Bh), 3 * g.N, s);
    for (int a = 0; a < 3; ++a) {
      Launch<T>::recon(g, recon, a, as<T>(c->W), as<T>(c->WL), as<T>(c->WR), s);
      Launch<T>::flux_hlld(g, a, as<T>(c->WL), as<T>(c->WR), as<T>(c->Bh), as<T>(c->F), s);
    }
  }
  Launch<T>::widen(as<T>(c->F), Fout, 21 * g.N, s);
  return cuda_status();
}

template <class T> int stage_edges(mhd_ctx* c, const double* U, const double* Fin, double* Eout) {
  const Grid& g = c->g;
  cudaStream_t s = c->stream;
  Launch<T>::prim(g, const_cast<double*>(U), as<T>(c->W), nullptr, c->flags, nullptr, s);
  Launch<T>::narrow(Fin, as<T>(c->F), 21 * g.N, s);
  Launch<T>::emf(g, as<T>(c->W), as<T>(c->F), as<T>(c->E), s);
  Launch<T>::widen(as<T>(c->E), Eout, 3 * g.N, s);
  return cuda_status();
}

template <class T> int stage_recon(mhd_ctx* c, const double* U, int axis, int recon, double* WL, double* WR) {
  const Grid& g = c->g;
  cudaStream_t s = c->stream;
  Launch<T>::prim(g, const_cast<double*>(U), as<T>(c->W), nullptr, c->flags, nullptr, s);
  Launch<T>::recon(g, recon, axis, as<T>(c->W), as<T>(c->WL), as<T>(c->WR), s);
  Launch<T>::widen(as<T>(c->WL), WL, 7 * g.N, s);
  Launch<T>::widen(as<T>(c->WR), WR, 7 * g.N, s);
  return cuda_status();
}

}  // namespace

extern "C" {

int mhd_workspace_bytes(const mhd_config* cfg, size_t* bytes) {
  int st = check_cfg(cfg);
  if (st != MHD_OK) return st;
  if (!bytes) return MHD_ERR_ARG;
  *bytes = layout_of(*cfg).total;
  return MHD_OK;
}

int mhd_init(mhd_ctx** out, const mhd_config* cfg, void* stream) {
  if (!out) return MHD_ERR_ARG;
  *out = nullptr;
  int st = check_cfg(cfg);
  if (st != MHD_OK) return st;
  mhd_ctx* c = new (std::nothrow) mhd_ctx();
  if (!c) return MHD_ERR_OOM;
  c->cfg = *cfg;
  int np[3], lo[3];
  padded_dims(*cfg, np, lo);
  for (int a = 0; a < 3; ++a) {
    c->g.n[a] = np[a];
    c->g.lo[a] = lo[a];
    c->g.hi[a] = np[a] - lo[a];
    c->g.bc[a] = MHD_BC_PERIODIC;  // the padded grid itself wraps
  }
  c->g.N = (long long)np[0] * np[1] * np[2];
  c->g.d[0] = cfg->dx;
  c->g.d[1] = cfg->dy;
  c->g.d[2] = cfg->dz;
  for (int a = 0; a < 3; ++a) c->g.id[a] = 1.0 / c->g.d[a];
  c->g.gm1 = cfg->gamma - 1.0;
  c->g.igm1 = 1.0 / (cfg->gamma - 1.0);
  c->g.gamma = cfg->gamma;
  c->g.rho_floor = cfg->rho_floor;
  c->g.p_floor = cfg->p_floor;
  c->g.cfl = cfg->cfl;
  c->gi = c->g;
  c->gi.n[0] = cfg->nx;
  c->gi.n[1] = cfg->ny;
  c->gi.n[2] = cfg->nz;
  c->gi.N = (long long)cfg->nx * cfg->ny * cfg->nz;
  for (int a = 0; a < 3; ++a) {
    c->gi.lo[a] = 0;
    c->gi.hi[a] = c->gi.n[a];
    c->gi.bc[a] = cfg->bc[a];
  }
  c->stream = static_cast<cudaStream_t>(stream);
  c->ts = cfg->precision == MHD_FP32_BULK ? 4 : 8;
  const Layout L = layout_of(*cfg);
  c->ws_bytes = L.total;
  cudaGetLastError();
  if (cudaMalloc(&c->ws, L.total) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return MHD_ERR_OOM;
  }
  char* b = static_cast<char*>(c->ws);
  c->W = b + L.W;
  c->F = b + L.F;
  c->E = b + L.E;
  c->WL = b + L.WL;
  c->WR = b + L.WR;
  c->Bh = b + L.Bh;
  c->Er = b + L.Er;
  c->scal = reinterpret_cast<double*>(b + L.scal);
  c->dtbits = reinterpret_cast<unsigned long long*>(b + L.dtbits);
  c->floors = reinterpret_cast<unsigned long long*>(b + L.floors);
  c->flags = reinterpret_cast<unsigned*>(b + L.flags);
  c->red = reinterpret_cast<double*>(b + L.red);
  c->red_count = red_blocks(c->gi.N);
  c->Up = padded(*cfg) ? reinterpret_cast<double*>(b + L.Up) : nullptr;
  cudaMemsetAsync(c->ws, 0, L.total, c->stream);
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
    cudaFree(c->ws);
    delete c;
    return MHD_ERR_CUDA;
  }
  *out = c;
  return MHD_OK;
}

void mhd_destroy(mhd_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->ws) cudaFree(c->ws);
  if (c->host_state) cudaFree(c->host_state);
  if (c->adj_ws) cudaFree(c->adj_ws);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
}

int mhd_profile_enable(mhd_ctx* c, int on) {
  if (!c) return MHD_ERR_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return MHD_ERR_CUDA;
  c->prof_on = on ? 1 : 0;
  c->prof.clear();
  c->ev_used = 0;
  return MHD_OK;
}

int mhd_profile_read(mhd_ctx* c, double ms[MHD_NUM_STAGES], long long launches[MHD_NUM_STAGES]) {
  if (!c || !ms || !launches) return MHD_ERR_ARG;
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return MHD_ERR_CUDA;
  for (int i = 0; i < MHD_NUM_STAGES; ++i) {
    ms[i] = 0;
    launches[i] = 0;
  }
  for (const ProfRec& r : c->prof) {
    float t = 0;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return MHD_ERR_CUDA;
    ms[r.stage] += t;
    launches[r.stage] += 1;
  }
  c->prof.clear();
  c->ev_used = 0;
  return MHD_OK;
}

const char* mhd_stage_name(int stage) {
  static const char* names[MHD_NUM_STAGES] = {"prim", "flux_pcm",    "emf", "update_half", "recon",
                                              "flux_hlld", "update_full", "dt",  "h2d",         "d2h"};
  if (stage < 0 || stage >= MHD_NUM_STAGES) return "unknown";
  return names[stage];
}

int mhd_step(mhd_ctx* c, double* U, double dt, double* next_dt_host) {
  if (!c || !U) return MHD_ERR_ARG;
  if (has_halo(c->cfg)) return MHD_ERR_ARG;  // subdomains step through mhd_step_sub
  if (!(dt > 0.0) || !std::isfinite(dt)) return MHD_ERR_DT;
  return with_type(c->cfg.precision, [&](auto t) { return one_step<MHD_T>(c, U, dt, next_dt_host); });
}

int mhd_floor_count(mhd_ctx* c, long long* n_rho, long long* n_p) {
  if (!c) return MHD_ERR_ARG;
  unsigned long long fc[2] = {0, 0};
  cudaStream_t s = c->stream;
  if (cudaMemcpyAsync(fc, c->floors, sizeof(fc), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ERR_CUDA;
  cudaMemsetAsync(c->floors, 0, 2 * sizeof(unsigned long long), s);
  if (n_rho) *n_rho = (long long)fc[0];
  if (n_p) *n_p = (long long)fc[1];
  return cuda_status();
}

int mhd_run(mhd_ctx* c, double* U, int nsteps, double* dt_dev) {
  if (!c || !U || nsteps < 0) return MHD_ERR_ARG;
  if (has_halo(c->cfg)) return MHD_ERR_ARG;  // subdomains step through mhd_step_sub
  if (nsteps == 0) return MHD_OK;
  return with_type(c->cfg.precision, [&](auto t) { return run_steps<MHD_T>(c, U, nsteps, dt_dev); });
}

int mhd_step_sub(mhd_ctx* c, const double* Ug, const int gn[3], const int off[3], double dt, double* Ug_out) {
  if (!c || !Ug || !gn || !off || !Ug_out || Ug == Ug_out || !has_halo(c->cfg)) return MHD_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return MHD_ERR_DT;
  const int st = check_sub(c, gn, off);
  if (st != MHD_OK) return st;
  return with_type(c->cfg.precision, [&](auto t) { return step_sub<MHD_T>(c, Ug, gn, off, dt, Ug_out); });
}

int mhd_dt_sub(mhd_ctx* c, const double* Ug, const int gn[3], const int off[3], double* dt_host) {
  if (!c || !Ug || !gn || !off || !dt_host || !has_halo(c->cfg)) return MHD_ERR_ARG;
  const int st = check_sub(c, gn, off);
  if (st != MHD_OK) return st;
  return with_type(c->cfg.precision, [&](auto t) { return dt_sub<MHD_T>(c, Ug, gn, off, dt_host); });
}

int mhd_evolve(mhd_ctx* c, double* U, double t_end, int max_steps, double* t_host, int* steps_host) {
  if (!c || !U || max_steps < 0 || !(t_end >= 0.0) || !std::isfinite(t_end)) return MHD_ERR_ARG;
  if (has_halo(c->cfg)) return MHD_ERR_ARG;
  return with_type(c->cfg.precision,
                   [&](auto t) { return evolve_to<MHD_T>(c, U, t_end, max_steps, t_host, steps_host); });
}

int mhd_dt(mhd_ctx* c, const double* U, double* dt_host) {
  if (!c || !U || !dt_host) return MHD_ERR_ARG;
  if (has_halo(c->cfg)) return MHD_ERR_ARG;  // subdomains step through mhd_step_sub
  cudaStream_t s = c->stream;
  cudaMemsetAsync(c->dtbits, 0, sizeof(unsigned long long), s);
  double* Um = enter(c, U);  // k_prim writes its state only when floors are requested
  with_type(c->cfg.precision, [&](auto t) {
    Launch<MHD_T>::prim(c->g, Um, as<MHD_T>(c->W), c->dtbits, c->flags, nullptr, s);
    return 0;
  });
  mhd::launch_finish_dt(c->g, c->dtbits, c->scal, nullptr, 0, c->flags, kNoEnd, s);
  double v = 0;
  unsigned fl = 0;
  if (cudaMemcpyAsync(&v, c->scal, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
  if (cudaMemcpyAsync(&fl, c->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ERR_CUDA;
  *dt_host = v;
  if (fl & 1u) return MHD_ERR_NONFINITE;
  if (!(v > 0.0) || !std::isfinite(v)) return MHD_ERR_DT;
  return MHD_OK;
}

int mhd_run_host(mhd_ctx* c, double* U_host, int nsteps, double* t_host) {
  if (!c || !U_host || nsteps < 0) return MHD_ERR_ARG;
  const size_t bytes = 8 * (size_t)c->gi.N * sizeof(double);
  if (!c->host_state) {
    if (cudaMalloc(&c->host_state, bytes) != cudaSuccess) {
      cudaGetLastError();
      c->host_state = nullptr;
      return MHD_ERR_OOM;
    }
  }
  cudaStream_t s = c->stream;
  cudaError_t e = cudaSuccess;
  prof(c, MHD_STAGE_H2D, [&] { e = cudaMemcpyAsync(c->host_state, U_host, bytes, cudaMemcpyHostToDevice, s); });
  if (e != cudaSuccess) return MHD_ERR_CUDA;
  int st = mhd_run(c, c->host_state, nsteps, nullptr);
  if (st != MHD_OK) return st;
  prof(c, MHD_STAGE_D2H, [&] { e = cudaMemcpyAsync(U_host, c->host_state, bytes, cudaMemcpyDeviceToHost, s); });
  if (e != cudaSuccess) return MHD_ERR_CUDA;
  double t = 0;
  if (cudaMemcpyAsync(&t, c->scal + 1, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ERR_CUDA;
  if (t_host) *t_host = t;
  return mhd_status(c, nullptr);
}

namespace {
// the kernel's transparent huge page size (PMD size), 2 MiB if not given
size_t huge_page_bytes() {
  size_t v = 0;
  if (FILE* f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
    unsigned long long x = 0;
    if (std::fscanf(f, "%llu", &x) == 1) v = (size_t)x;
    std::fclose(f);
  }
  return (v >= 4096 && (v & (v - 1)) == 0) ? v : ((size_t)2 << 20);
}
}  // namespace

int mhd_host_alloc(size_t bytes, void** out) {
  if (!out || bytes == 0) return MHD_ERR_ARG;
  *out = nullptr;
  // huge pages for buffers of at least a quarter huge page (a state of 8.6 GB
  // is 17 pages of 512 MiB); smaller ones are page-aligned
  const size_t hp_sys = huge_page_bytes();
  const size_t hp = bytes >= hp_sys / 4 ? hp_sys : (size_t)4096;
  if (bytes > SIZE_MAX - hp) return MHD_ERR_ARG;
  const size_t total = (bytes + hp - 1) / hp * hp;
  void* p = nullptr;
  if (posix_memalign(&p, hp, total) != 0 || !p) return MHD_ERR_OOM;
#ifdef MADV_HUGEPAGE
  if (hp == hp_sys) madvise(p, total, MADV_HUGEPAGE);  // advice only: without huge pages the memory stays usable
#endif
  if (cudaHostRegister(p, total, cudaHostRegisterDefault) != cudaSuccess) {
    cudaGetLastError();
    std::free(p);
    return MHD_ERR_CUDA;
  }
  *out = p;
  return MHD_OK;
}

int mhd_host_free(void* p) {
  if (!p) return MHD_OK;
  if (cudaHostUnregister(p) != cudaSuccess) {
    cudaGetLastError();
    return MHD_ERR_CUDA;
  }
  std::free(p);
  return MHD_OK;
}

int mhd_adjoint_step(mhd_ctx* c, const double* U_n, double dt, const double* gU_np1, double* gU_n) {
  if (!c || !U_n || !gU_np1 || !gU_n || gU_np1 == gU_n) return MHD_ERR_ARG;
  if (c->cfg.recon == MHD_RECON_PLM_PRIM) return MHD_ERR_ARG;  // no reverse sweep for this variant
  if (c->Up) return MHD_ERR_ARG;  // periodic grids only
  if (!(dt > 0.0) || !std::isfinite(dt)) return MHD_ERR_DT;
  return with_adj_type(c->cfg.precision, [&](auto t) { return adjoint_step<MHD_T>(c, U_n, dt, gU_np1, gU_n); });
}

int mhd_adjoint_step_cfl(mhd_ctx* c, const double* U_n, const double* gU_np1, double* gU_n, double* dt_host,
                         double* g_dt_host) {
  if (!c || !U_n || !gU_np1 || !gU_n || gU_np1 == gU_n) return MHD_ERR_ARG;
  if (c->cfg.recon == MHD_RECON_PLM_PRIM) return MHD_ERR_ARG;
  if (c->Up) return MHD_ERR_ARG;
  return with_adj_type(c->cfg.precision, [&](auto t) {
    return adjoint_step<MHD_T>(c, U_n, 0.0, gU_np1, gU_n, true, dt_host, g_dt_host);
  });
}

int mhd_adjoint_workspace_bytes(const mhd_config* cfg, size_t* bytes) {
  int st = check_cfg(cfg);
  if (st != MHD_OK) return st;
  if (!bytes) return MHD_ERR_ARG;
  *bytes = adj_bytes_of(*cfg);
  return MHD_OK;
}

int mhd_stage_recon_vjp(mhd_ctx* c, const double* U, int axis, int recon, const double* gWL, const double* gWR,
                        double* gU) {
  if (!c || !U || !gWL || !gWR || !gU || axis < 0 || axis > 2 || recon < MHD_RECON_PCM || recon > MHD_RECON_PPMC)
    return MHD_ERR_ARG;
  if (c->Up) return MHD_ERR_ARG;  // periodic grids only
  return with_adj_type(c->cfg.precision,
                       [&](auto t) { return stage_recon_vjp<MHD_T>(c, U, axis, recon, gWL, gWR, gU); });
}

int mhd_stage_hlld_vjp(int n, double gamma, int precision, const double* wl, const double* wr, const double* bn,
                       const double* gf, double* gwl, double* gwr, double* gbn, double* f, void* stream) {
  if (n < 0 || !wl || !wr || !bn || !gf || !gwl || !gwr || !gbn || !f || !(gamma > 1.0)) return MHD_ERR_ARG;
  if (n == 0) return MHD_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  with_type(precision, [&](auto t) {
    mhd::AdjLaunch<MHD_T>::hlld_batch(n, gamma, wl, wr, bn, gf, gwl, gwr, gbn, f, s);
    return 0;
  });
  return cuda_status();
}

int mhd_status(mhd_ctx* c, long long counts[2]) {
  if (!c) return MHD_ERR_ARG;
  unsigned fl = 0;
  unsigned long long fc[2] = {0, 0};
  cudaStream_t s = c->stream;
  if (cudaMemcpyAsync(&fl, c->flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
  if (cudaMemcpyAsync(fc, c->floors, sizeof(fc), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ERR_CUDA;
  cudaMemsetAsync(c->flags, 0, sizeof(unsigned), s);
  cudaMemsetAsync(c->floors, 0, 2 * sizeof(unsigned long long), s);
  if (counts) {
    counts[0] = (long long)fc[0];
    counts[1] = (long long)fc[1];
  }
  if (fl & 1u) return MHD_ERR_NONFINITE;
  if (fl & 2u) return MHD_ERR_DT;
  return MHD_OK;
}

const char* mhd_strerror(int code) {
  switch (code) {
    case MHD_OK: return "ok";
    case MHD_ERR_ARG: return "invalid argument";
    case MHD_ERR_CUDA: return "CUDA runtime error";
    case MHD_ERR_OOM: return "out of device memory";
    case MHD_ERR_NONFINITE: return "non-finite value or non-positive density in the state";
    case MHD_ERR_DT: return "time step not positive or not finite";
    case MHD_ERR_TOO_LARGE: return "grid larger than the 17.8 MB static scratch of mhd_diagnostics_static (512^3 cells)";
    default: return "unknown status";
  }
}

int mhd_diagnostics(mhd_ctx* c, const double* U, double* divb_max, double totals[8]) {
  if (!c || !U || !divb_max || !totals) return MHD_ERR_ARG;
  cudaStream_t s = c->stream;
  mhd::launch_diagnostics(c->gi, U, c->red, (int)c->red_count, s);
  double out[9];
  if (cudaMemcpyAsync(out, c->red, sizeof(out), cudaMemcpyDeviceToHost, s) != cudaSuccess) return MHD_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MHD_ERR_CUDA;
  *divb_max = out[8];
  for (int f = 0; f < 8; ++f) totals[f] = out[f];
  return MHD_OK;
}


int mhd_stage_primitives(mhd_ctx* c, const double* U, double* W) {
  if (!c || !U || !W) return MHD_ERR_ARG;
  if (c->Up) return MHD_ERR_ARG;  // periodic grids only
  return with_type(c->cfg.precision, [&](auto t) { return stage_prims<MHD_T>(c, U, W); });
}



int mhd_stage_fluxes(mhd_ctx* c, const double* U, int recon, double* F) {
  if (!c || !U || !F || recon < MHD_RECON_PCM || recon > MHD_RECON_PLM_PRIM) return MHD_ERR_ARG;
  if (c->Up) return MHD_ERR_ARG;  // periodic grids only
  return with_type(c->cfg.precision, [&](auto t) { return stage_fluxes<MHD_T>(c, U, recon, F); });
}



int mhd_stage_edges(mhd_ctx* c, const double* U, const double* F, double* E) {
  if (!c || !U || !F || !E) return MHD_ERR_ARG;
  if (c->Up) return MHD_ERR_ARG;  // periodic grids only
  return with_type(c->cfg.precision, [&](auto t) { return stage_edges<MHD_T>(c, U, F, E); });
}



int mhd_stage_recon(mhd_ctx* c, const double* U, int axis, int recon, double* WL, double* WR) {
  if (!c || !U || !WL || !WR || axis < 0 || axis > 2 || recon < MHD_RECON_PCM || recon > MHD_RECON_PLM_PRIM)
    return MHD_ERR_ARG;
  if (c->Up) return MHD_ERR_ARG;  // periodic grids only
  return with_type(c->cfg.precision, [&](auto t) { return stage_recon<MHD_T>(c, U, axis, recon, WL, WR); });
}


}  // extern "C"
