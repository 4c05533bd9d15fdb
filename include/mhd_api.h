/* mhd_api.h -- C ABI of the GB300 VL+CT ideal-MHD library (libmhd.so).
 *
 * Method: the Van Leer + Constrained Transport step of Caddy & Schneider,
 * "Cholla-MHD" (arXiv:2402.05240), Sec. 2.2, Steps 1-10: CFL time step
 * (Eq. dt), PCM predictor fluxes from the HLLD Riemann solver (Steps 2-3),
 * edge electric fields (Eq. emf-edge, Steps 4 and 8), half-step update
 * (Step 5), PLMC/PPMC characteristic reconstruction (Step 6, Sec. 2.2.6),
 * corrector fluxes (Step 7) and full-step update (Step 9), on a 3-D Cartesian
 * mesh, periodic by default (outflow boundaries and halo-fed subdomains are
 * options of mhd_config).
 *
 * State layout (all entry points): one contiguous float64 array
 *   U[8][nz][ny][nx], x fastest, fields rho, mx, my, mz, E, Bx, By, Bz
 * (the conserved vector U of Sec. 2.1).  Bx[k][j][i] is the face-centred
 * field at x_{i+1/2} (the upper x-face of cell i; Sec. 2.2 "staggered grid");
 * By at y_{j+1/2}, Bz at z_{k+1/2}.  The caller's arrays hold no ghost
 * cells: periodic neighbours are found by wrap-around indexing inside the
 * kernels, and outflow axes are padded inside the library's workspace.
 *
 * Pointers: arguments named *_dev are device pointers (cudaMalloc / torch
 * CUDA tensors), *_host host pointers.  The caller owns every state and
 * gradient buffer.  The library owns the workspace it allocates in
 * mhd_init, the adjoint workspace and the device copy of mhd_run_host that
 * it allocates on first use, all freed by mhd_destroy, and the static
 * scratch of mhd_diagnostics_static.  All device work of a context is
 * issued on the stream given to mhd_init (NULL = legacy default stream).
 * A context holds mutable host state (profiling records, the lazily
 * allocated buffers): calls on one context from several host threads must
 * be serialised by the caller; separate contexts are independent.
 *
 * Errors: every call except mhd_destroy, mhd_strerror and mhd_stage_name
 * returns an int status (MHD_OK = 0, negative on error); the library never
 * exits, aborts or traps.  Device kernels raise flags
 * (non-finite value, non-positive density) that the synchronising calls
 * (mhd_dt, mhd_status, mhd_diagnostics, mhd_run_host) report.
 */
#ifndef MHD_API_H
#define MHD_API_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MHD_OK 0
#define MHD_ERR_ARG (-1)       /* invalid argument (NULL, size, option)        */
#define MHD_ERR_CUDA (-2)      /* a CUDA runtime call failed                   */
#define MHD_ERR_OOM (-3)       /* workspace allocation failed                  */
#define MHD_ERR_NONFINITE (-4) /* a kernel saw NaN/Inf or density <= 0         */
#define MHD_ERR_DT (-5)        /* dt <= 0 or not finite                        */
#define MHD_ERR_TOO_LARGE (-6) /* grid above the static scratch of mhd_diagnostics_static */

#define MHD_RECON_PCM 0  /* piecewise constant (Sec. 2.2.2)                   */
#define MHD_RECON_PLMC 1 /* piecewise linear, characteristic (Sec. 2.2.6)     */
#define MHD_RECON_PPMC 2 /* piecewise parabolic, characteristic (Felker & Stone 2018) */
#define MHD_RECON_PLM_PRIM 3 /* piecewise linear limited in the primitive variables
                                (Sec. 2.2.6, last paragraph); no adjoint */

#define MHD_FP64 0      /* all arithmetic in float64                          */
#define MHD_FP32_BULK 1 /* reconstruction, Riemann solver and EMFs in float32;
                           state accumulation and pressure recovery in float64 */
#define MHD_FP64_DF 2   /* reconstruction, Riemann solver, EMFs and the update
                           increments in double-float (a float pair, ~2^-47
                           relative error per operation, float exponent range)
                           on the FP32 pipes; state, pressure recovery and
                           accumulation in float64.  Differs from MHD_FP64 at
                           the 1e-13 level; so does its adjoint (reverse sweep
                           in double-float, cotangents of the state in
                           float64). */

/* Boundary condition of each axis (mhd_config.bc).  Periodic: wrap-around
 * indexing inside the kernels, no ghost cells.  Outflow (zero gradient, the
 * paper's Riemann problems, Sec. 3.1.4): the library embeds the grid in a
 * padded grid with MHD_GHOST cells on both sides of each outflow axis, fills
 * every ghost cell (all 8 fields, face fields included) from the nearest
 * interior cell before each step, and runs the step on the padded grid; the
 * ghost depth exceeds the step's dependency radius (5 cells for PPMC), so
 * the interior result is that of ghost cells filled once per step.  The CFL
 * dt and the floor counters cover interior cells only. */
#define MHD_BC_PERIODIC 0
#define MHD_BC_OUTFLOW 1
#define MHD_BC_HALO 2 /* subdomain of a decomposed periodic grid: MHD_GHOST halo
                         cells per side, filled by mhd_step_sub (only entry
                         point that accepts it) */
#define MHD_GHOST 8

typedef struct mhd_config {
  int nx, ny, nz;          /* cells per axis, each >= 4; nz <= 65535 and at
                              most 2^31 - 1 cells in all (with the ghost
                              cells of outflow and halo axes)               */
  double dx, dy, dz;       /* cell widths (> 0)                               */
  double gamma;            /* adiabatic index, P = (gamma-1) eps (Sec. 2.1)   */
  double cfl;              /* Courant number C_CFL of Eq. dt (0 < cfl <= 0.5) */
  int recon;               /* MHD_RECON_* for Step 6                          */
  int precision;           /* MHD_FP64, MHD_FP32_BULK or MHD_FP64_DF          */
  double rho_floor;        /* density floor (use 1e-20 for "off")             */
  double p_floor;          /* pressure floor (use 1e-20 for "off")            */
  int bc[3];               /* MHD_BC_* per axis x, y, z                       */
} mhd_config;

typedef struct mhd_ctx mhd_ctx; /* opaque; owns the workspace */

/* Library infrastructure, not in the paper.  *bytes receives the device
 * workspace mhd_init allocates for cfg (primitives, fluxes, edge fields,
 * reconstructed states, scratch of the reductions; sized for the compute
 * type of cfg->precision).  No device work.  Errors: MHD_ERR_ARG (cfg or
 * bytes NULL, or cfg invalid). */
int mhd_workspace_bytes(const mhd_config* cfg, size_t* bytes);

/* Library infrastructure, not in the paper.  Creates a context for cfg on
 * the current CUDA device; stream is a cudaStream_t (NULL = default stream)
 * that every later call on the context uses.  Allocates and zeroes the
 * workspace (mhd_workspace_bytes) and synchronises the stream.  *out
 * receives the context (owned by the caller, freed by mhd_destroy), or NULL
 * on error.  Errors: MHD_ERR_ARG (out or cfg NULL, cfg invalid),
 * MHD_ERR_OOM (host or device allocation failed), MHD_ERR_CUDA. */
int mhd_init(mhd_ctx** out, const mhd_config* cfg, void* stream);

/* Library infrastructure, not in the paper.  Synchronises the context's
 * stream, then frees the workspace, the adjoint workspace, the device copy
 * used by mhd_run_host, the profiling events and the context itself; the
 * stream is the caller's and is not destroyed.  NULL is ignored. */
void mhd_destroy(mhd_ctx* ctx);

/* Step 1, Eq. dt: dt = C_CFL * min over cells and directions l of
 * d_l / (|v_l| + c_f,l), c_f from cell-centred values with longitudinal B_l.
 * U_dev: state (read only).  Synchronous; writes the value to *dt_host. */
int mhd_dt(mhd_ctx* ctx, const double* U_dev, double* dt_host);

/* One VL+CT step (Steps 2-9) at the given dt, in place: U_dev holds U^n on
 * entry and U^{n+1} on return.  Asynchronous on the context's stream when
 * next_dt_host is NULL; otherwise the CFL dt of U^{n+1} (Step 1 of the next
 * step, from the same pass that applies the floors) is written there and the
 * call synchronises (MHD_ERR_DT if it is not positive and finite). */
int mhd_step(mhd_ctx* ctx, double* U_dev, double dt, double* next_dt_host);

/* nsteps VL+CT steps, each with dt from Step 1 computed on the device (the
 * reduction of the full update of one step gives the dt of the next), in
 * place.  dt_dev (device, may be NULL) receives the nsteps dt values used.
 * Asynchronous. */
int mhd_run(mhd_ctx* ctx, double* U_dev, int nsteps, double* dt_dev);

/* One step (Steps 2-10 at the given dt) of a subdomain of a periodic global
 * grid: domain decomposition (Step 10 exchanges the halo cells of each
 * rank's subdomain; Sec. 3.2 runs one subdomain per GPU).  ctx:
 * created with cfg.nx, ny, nz = the subdomain's cells and bc = MHD_BC_HALO
 * on every decomposed axis (MHD_BC_PERIODIC on axes it spans whole).
 * Ug_dev: a state [8][gn[2]][gn[1]][gn[0]] holding the subdomain at offset
 * off[3] and at least MHD_GHOST cells of halo around it along the decomposed
 * axes (a whole periodic global grid, wrapped, or the subdomain's own
 * halo-extended block at offset MHD_GHOST); read only.  Ug_out_dev (must not
 * alias Ug_dev): receives the subdomain's new interior at the same offset;
 * other cells are untouched.  The interior equals that of one mhd_step on
 * the whole global grid bit for bit.  Asynchronous.  Errors: MHD_ERR_ARG
 * (no MHD_BC_HALO axis, sizes, offsets, aliasing), MHD_ERR_DT. */
int mhd_step_sub(mhd_ctx* ctx, const double* Ug_dev, const int gn[3], const int off[3], double dt, double* Ug_out_dev);

/* Step 1 (Eq. dt) over the interior cells of a subdomain, with Ug_dev, gn
 * and off as in mhd_step_sub (the halo supplies the lower faces of the first
 * cells).  Synchronous; the global dt is the minimum over the subdomains. */
int mhd_dt_sub(mhd_ctx* ctx, const double* Ug_dev, const int gn[3], const int off[3], double* dt_host);

/* Advance U_dev in place from t = 0 to t = t_end (the end time of the paper's
 * tests, Sec. 3): device-dt steps as in mhd_run, the last one shortened so
 * that it lands on t_end exactly; at most max_steps steps.  Reads the time
 * back after each step (synchronous).  *t_host (may be NULL) receives the
 * time reached (t_end unless max_steps ran out), *steps_host (may be NULL)
 * the steps taken.  Errors: MHD_ERR_ARG (t_end < 0 or not finite,
 * max_steps < 0), MHD_ERR_NONFINITE / MHD_ERR_DT from the device flags, the
 * state then holds the step that raised them. */
int mhd_evolve(mhd_ctx* ctx, double* U_dev, double t_end, int max_steps, double* t_host, int* steps_host);

/* Steps 1-9 (Sec. 2.2) as in mhd_run, on a HOST state (not in the paper:
 * the end-to-end form that includes the host<->device copies).  U_host
 * (8 x N doubles, layout as U_dev; pinned memory for full copy bandwidth):
 * copied to a device buffer the context allocates on the first call and
 * keeps, stepped nsteps times in place, copied back; synchronous.  *t_host
 * (may be NULL) receives the simulated time advanced (the sum of the dt
 * values).  Errors: MHD_ERR_ARG (ctx or U_host NULL, nsteps < 0, a
 * subdomain context), MHD_ERR_OOM, MHD_ERR_CUDA, then the device flags as
 * mhd_status returns them. */
int mhd_run_host(mhd_ctx* ctx, double* U_host, int nsteps, double* t_host);

/* Library infrastructure, not in the paper.  Allocates bytes of
 * page-locked host memory for mhd_run_host (or any host<->device copy):
 * from a quarter of the transparent huge page size up (2 MiB or 512 MiB,
 * from the kernel; 2 MiB if it does not say), aligned to and rounded up to a
 * multiple of that size and advised as huge pages; smaller requests page
 * aligned.  The memory is then registered with cudaHostRegister on the
 * current device.
 * On hosts whose DMA reaches host memory through an IOMMU (the Grace host of
 * a GB300), copies from ordinary page-locked memory slow down to a fraction
 * of the link rate after GPU work has run in between (translation misses
 * over the many small pages), while copies from huge-page memory keep the
 * full rate.  Where the kernel gives no huge pages, the memory is ordinary
 * page-locked memory.  *out_host receives the address (owned by the caller,
 * freed by mhd_host_free; contents undefined).  No device work.  Errors:
 * MHD_ERR_ARG (out_host NULL or bytes 0), MHD_ERR_OOM (host allocation
 * failed), MHD_ERR_CUDA (registration failed, e.g. no CUDA device). */
int mhd_host_alloc(size_t bytes, void** out_host);

/* Library infrastructure, not in the paper.  Unregisters and frees memory
 * from mhd_host_alloc (NULL: no-op).  Errors: MHD_ERR_CUDA (unregistration
 * failed; the memory is not freed). */
int mhd_host_free(void* host);

/* Vector-Jacobian product of one mhd_step at fixed dt (not in the paper):
 * gU_n = (dU^{n+1}/dU^n)^T gU_np1.  U_n_dev: the state the forward step
 * started from (read only); gU_np1_dev: cotangent of U^{n+1}; gU_n_dev:
 * output, same layout as U.  Recomputes the forward intermediates in the
 * workspace.  Asynchronous.  Periodic grids and MHD_RECON_PCM / PLMC / PPMC
 * only (MHD_ERR_ARG otherwise). */
int mhd_adjoint_step(mhd_ctx* ctx, const double* U_n_dev, double dt, const double* gU_np1_dev,
                     double* gU_n_dev);

/* Vector-Jacobian product of one step whose dt is the CFL dt of its own
 * start state (not in the paper): U^{n+1} = S(U^n, dt(U^n)) with
 * dt(U) = C_CFL / max over cells and axes of (|v_l| + c_f,l) / d_l (Eq. dt,
 * Step 1), so gU_n = (dS/dU^n)^T gU_np1 + g_dt (d dt/dU^n)^T with
 * g_dt = <gU_np1, dS/d dt>.  The maximum is differentiated at the lowest
 * cell index that reaches it (then the lowest axis): one element of the
 * subdifferential where cells tie.  Arguments as in mhd_adjoint_step;
 * *dt_host and *g_dt_host (each may be NULL) receive dt (the value mhd_dt
 * returns for U_n) and g_dt.  Synchronous (dt is read back before the
 * recompute).  Errors: as mhd_adjoint_step, MHD_ERR_NONFINITE /
 * MHD_ERR_DT from the reduction. */
int mhd_adjoint_step_cfl(mhd_ctx* ctx, const double* U_n_dev, const double* gU_np1_dev, double* gU_n_dev,
                         double* dt_host, double* g_dt_host);

/* Library infrastructure of the adjoint (not in the paper).  *bytes
 * receives the device memory the first mhd_adjoint_step or
 * mhd_adjoint_step_cfl call allocates (once per context, freed by
 * mhd_destroy): forward intermediates of one step plus cotangent buffers,
 * 148 words of the compute type (a float pair for MHD_FP64_DF) + 10
 * doubles per cell, plus the partials of the CFL reduction.  The adjoint
 * also uses 49 words per cell of the context's step workspace
 * (mhd_workspace_bytes), whose contents no call relies on between calls.  No
 * device work.  Errors: MHD_ERR_ARG (cfg or bytes NULL, or cfg invalid). */
int mhd_adjoint_workspace_bytes(const mhd_config* cfg, size_t* bytes);

/* Diagnostics of a state (Sec. 3, div B at round-off): max over cells of
 * |div B| from face differences, and the sums of the 8 fields.  On an
 * outflow axis the lower face of the first cell is its ghost copy (equal to
 * the cell's upper face).  Synchronous. */
int mhd_diagnostics(mhd_ctx* ctx, const double* U_dev, double* divb_max_host, double totals_host[8]);

/* mhd_diagnostics without any device allocation.  The paper has no
 * counterpart: this serves callers that cannot call cudaMalloc -- a host
 * whose device memory is already owned by another allocator, or a step loop
 * that must not pay the implicit synchronisation of cudaMalloc/cudaFree.
 * It needs no context: cfg supplies nx, ny, nz (>= 1 each) and dx, dy, dz;
 * U_dev is a state in the usual layout; the work runs on `stream` (a
 * cudaStream_t, NULL = default stream) and the call synchronises it before
 * writing the max |div B| and the 8 field sums to host memory.
 * Scratch: a file-scope device array of 17.8 MB (9 results, then 9 partial
 * values and 8 compensation terms per 1024-cell block: 9 + 17 * 131072
 * doubles for grids up to 512^3 = 134,217,728 cells) that every GPU loading
 * the library holds until the process exits.  Larger grids return
 * MHD_ERR_TOO_LARGE.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  The address is cached per device
 * ordinal for the life of the process and is not looked up again after a
 * cudaDeviceReset: do not call this after resetting a device.
 * All calls share the one array and it keeps the last call's contents:
 * calls whose work overlaps on the GPU (other streams, other host threads
 * on the same device) race and must be serialised by the caller. */
int mhd_diagnostics_static(const mhd_config* cfg, const double* U_dev, void* stream, double* divb_max_host,
                           double totals_host[8]);

/* Library infrastructure, not in the paper.  Synchronises the context's
 * stream and reads the device flags raised since the last call, then clears
 * them; counts_host[0..1] (may be NULL) receive the density / pressure
 * floor triggers (Sec. 2.2 floors, reading D-12) of the full updates since
 * the last call, then reset.  Returns MHD_ERR_NONFINITE (a non-finite value
 * or a non-positive density was seen), else MHD_ERR_DT (a device dt that
 * was not positive and finite), else MHD_OK; MHD_ERR_ARG for a NULL ctx,
 * MHD_ERR_CUDA if the stream failed. */
int mhd_status(mhd_ctx* ctx, long long counts_host[2]);

/* The density / pressure floors of the full update (Sec. 2.2, reading
 * D-12: cells whose density or pressure fell below cfg.rho_floor /
 * cfg.p_floor and were reset).  Synchronises the context's stream;
 * *n_rho_host and *n_p_host (each may be NULL) receive the triggers since
 * the last call of this function or of mhd_status, which are then reset;
 * the error flags are left for mhd_status.  Errors: MHD_ERR_ARG (NULL
 * ctx), MHD_ERR_CUDA. */
int mhd_floor_count(mhd_ctx* ctx, long long* n_rho_host, long long* n_p_host);

/* Library infrastructure, not in the paper.  A static, NUL-terminated
 * English message for a status code ("unknown status" for codes the library
 * does not return); never NULL, never to be freed. */
const char* mhd_strerror(int code);

/* ---- tracing: per-stage CUDA-event timing -----------------------------
 * With profiling on, every kernel launch of mhd_run / mhd_step is bracketed
 * by CUDA events on the context's stream; mhd_profile_read synchronises and
 * returns, per stage, the summed device milliseconds and the launch count
 * since the last enable/read (then clears them).  Stage ids: */
#define MHD_STAGE_PRIM 0        /* primitives, floors, dt reduction (Step 1) */
#define MHD_STAGE_FLUX_PCM 1    /* PCM + HLLD predictor fluxes (Steps 2-3)    */
#define MHD_STAGE_EMF 2         /* edge electric fields (Steps 4, 8)          */
#define MHD_STAGE_UPDATE_HALF 3 /* half-step update (Step 5)                  */
#define MHD_STAGE_RECON 4       /* PLMC / PPMC states (Step 6)                */
#define MHD_STAGE_FLUX_HLLD 5   /* corrector HLLD fluxes (Step 7)             */
#define MHD_STAGE_UPDATE_FULL 6 /* full-step update (Step 9)                  */
#define MHD_STAGE_DT 7          /* dt finalisation                            */
#define MHD_STAGE_H2D 8         /* host -> device copy of mhd_run_host        */
#define MHD_STAGE_D2H 9         /* device -> host copy of mhd_run_host        */
#define MHD_NUM_STAGES 10

/* Library infrastructure, not in the paper.  Synchronises the context's
 * stream, turns the per-stage timing on (on != 0) or off and clears what
 * was recorded.  Errors: MHD_ERR_ARG (NULL ctx), MHD_ERR_CUDA. */
int mhd_profile_enable(mhd_ctx* ctx, int on);

/* Library infrastructure, not in the paper.  Synchronises the context's
 * stream; ms_host[s] receives the summed device milliseconds and
 * launches_host[s] the launch count of stage s since the last enable or
 * read (both zero with profiling off); the record is then cleared.
 * Errors: MHD_ERR_ARG (a NULL argument), MHD_ERR_CUDA. */
int mhd_profile_read(mhd_ctx* ctx, double ms_host[MHD_NUM_STAGES], long long launches_host[MHD_NUM_STAGES]);

/* Library infrastructure, not in the paper.  A static short name of a stage
 * id ("prim", "flux_pcm", ...; "unknown" out of range); never NULL. */
const char* mhd_stage_name(int stage);

/* ---- per-stage entry points (for stage-by-stage parity checks) ---------
 * All outputs are float64 device arrays in the oracle's layouts; in
 * MHD_FP32_BULK and MHD_FP64_DF modes the intermediates are widened on
 * output.  Periodic grids only (MHD_ERR_ARG otherwise). */

/* W_dev[8][N]: rho, vx, vy, vz, P, Bcc_x, Bcc_y, Bcc_z (Sec. 2.2.1). */
int mhd_stage_primitives(mhd_ctx* ctx, const double* U_dev, double* W_dev);

/* F_dev[3][7][N]: HLLD flux through the upper face of every cell per axis
 * a, in the solver frame (rho, m_n, m_t1, m_t2, E, B_t1, B_t2) with
 * (n, t1, t2) = (a, a+1, a+2) cyclically; states from recon (Steps 2-3, 6-7). */
int mhd_stage_fluxes(mhd_ctx* ctx, const double* U_dev, int recon, double* F_dev);

/* E_dev[3][N]: edge field E_a of every cell at p + e_b/2 + e_c/2 from the
 * fluxes F_dev and the reference fields of U_dev (Eq. emf-edge, Step 4). */
int mhd_stage_edges(mhd_ctx* ctx, const double* U_dev, const double* F_dev, double* E_dev);

/* WL_dev/WR_dev[7][N]: W_{L,p+1/2} and W_{R,p-1/2} of every cell along axis
 * (Step 6), solver frame, for recon = MHD_RECON_*. */
int mhd_stage_recon(mhd_ctx* ctx, const double* U_dev, int axis, int recon, double* WL_dev, double* WR_dev);

/* Vector-Jacobian product of the map U -> (W_L, W_R) of one axis (primitive
 * recovery, Sec. 2.2.1, then the reconstruction of Step 6): given the
 * cotangents gWL_dev, gWR_dev [7][N] (layouts of mhd_stage_recon), writes
 * gU_dev [8][N].  Uses the adjoint workspace. */
int mhd_stage_recon_vjp(mhd_ctx* ctx, const double* U_dev, int axis, int recon, const double* gWL_dev,
                        const double* gWR_dev, double* gU_dev);

/* HLLD flux and its vector-Jacobian product on n independent faces (Step 3;
 * Miyoshi & Kusano 2005): wl_dev, wr_dev [n][7] solver-frame primitive states
 * (rho, u, v, w, P, B_t1, B_t2), bn_dev [n] longitudinal fields, gf_dev [n][7]
 * flux cotangents; writes gwl_dev, gwr_dev [n][7], gbn_dev [n] and the flux
 * f_dev [n][7].  precision: MHD_FP64, MHD_FP32_BULK (arithmetic in float) or
 * MHD_FP64_DF (float pairs).
 * No context needed; asynchronous on stream. */
int mhd_stage_hlld_vjp(int n, double gamma, int precision, const double* wl_dev, const double* wr_dev,
                       const double* bn_dev, const double* gf_dev, double* gwl_dev, double* gwr_dev, double* gbn_dev,
                       double* f_dev, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* MHD_API_H */
