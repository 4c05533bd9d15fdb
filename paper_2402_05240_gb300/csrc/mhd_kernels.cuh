// mhd_kernels.cuh -- the kernels of one VL+CT step and their launchers.
//
// Schedule of one step (Caddy & Schneider, arXiv:2402.05240, Sec. 2.2):
//   k_prim          Step 1: primitives W^n (+ CFL dt min-reduction)
//   k_flux_pcm<A>   Steps 2-3: PCM states + HLLD on the faces of axis A
//   k_emf           Step 4: edge electric fields (reference fields of W^n)
//   k_update_half   Step 5: U^{n+1/2}, B^{n+1/2}; emits W^{n+1/2} and the
//                   half-step face fields (the hydro U^{n+1/2} is never stored)
//   k_recon<DIR>    Step 6: PLMC / PPMC interface states per axis
//   k_flux_hlld     Step 7: HLLD on the reconstructed states
//   k_emf           Step 8: edge fields with the half-step reference fields
//   k_update_full   Step 9: U^{n+1}, B^{n+1} in place
//   k_prim (floors) end of step: floors, W^{n+1} and the dt of the next step
// Periodic boundaries are wrapped neighbour offsets inside every kernel (each
// thread forms its six once: thread_cell); no ghost cells exist.  Threads map
// to cells with x fastest (coalesced rows), with 32-bit cell indices.
#pragma once

#include <type_traits>

#include "mhd_device.cuh"

namespace mhd {

struct CellIdx {
  int i, j, k;
  bool ok;
};

__device__ __forceinline__ CellIdx cell_of_thread(const Grid& g) {
  CellIdx c;
  c.i = blockIdx.x * BX + threadIdx.x;
  c.j = blockIdx.y * BY + threadIdx.y;
  c.k = blockIdx.z;
  c.ok = c.i < g.n[0] && c.j < g.n[1];
  return c;
}

inline dim3 grid_of(const Grid& g) { return dim3((g.n[0] + BX - 1) / BX, (g.n[1] + BY - 1) / BY, g.n[2]); }

// inside the interior box of a padded grid (always true without padding)
__device__ __forceinline__ bool interior(const Grid& g, int i, int j, int k) {
  return i >= g.lo[0] && i < g.hi[0] && j >= g.lo[1] && j < g.hi[1] && k >= g.lo[2] && k < g.hi[2];
}

// ------------------------------------------------------- 32-bit addressing --
// The step kernels address cells with 32-bit indices: every grid of a context
// has fewer than 2^31 cells (mhd_init refuses larger ones).  A thread forms
// its cell index and the periodic offsets to its six face neighbours once;
// any other stencil cell is the index plus a sum of offsets (the wrap along
// one axis does not depend on the other coordinates).  Field-major arrays
// reach the kernels as tables of field pointers (kernel parameters), so the
// address of field f at cell q is one 32 x 64-bit multiply-add: no 64-bit
// index arithmetic per access.
struct Cell {
  int i, j, k;
  int c;           // (k ny + j) nx + i
  int m[3], p[3];  // c + m[a]: the cell p - e_a, c + p[a]: the cell p + e_a (periodic)
  bool ok;
};

__device__ __forceinline__ Cell thread_cell(const Grid& g) {
  Cell p;
  p.i = blockIdx.x * BX + threadIdx.x;
  p.j = blockIdx.y * BY + threadIdx.y;
  p.k = blockIdx.z;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxy = nx * ny;
  p.ok = p.i < nx && p.j < ny;
  p.c = (p.k * ny + p.j) * nx + p.i;
  p.m[0] = p.i == 0 ? nx - 1 : -1;
  p.p[0] = p.i == nx - 1 ? 1 - nx : 1;
  p.m[1] = p.j == 0 ? (ny - 1) * nx : -nx;
  p.p[1] = p.j == ny - 1 ? (1 - ny) * nx : nx;
  p.m[2] = p.k == 0 ? (nz - 1) * nxy : -nxy;
  p.p[2] = p.k == nz - 1 ? (1 - nz) * nxy : nxy;
  return p;
}

// offset from cell p to p + s e_A (periodic), |s| < n[A]
template <int A> __device__ __forceinline__ int off(const Grid& g, const Cell& p, int s) {
  if (s == 0) return 0;
  if (s == -1) return p.m[A];
  if (s == 1) return p.p[A];
  const int x = A == 0 ? p.i : (A == 1 ? p.j : p.k);
  const int stride = A == 0 ? 1 : (A == 1 ? g.n[0] : g.n[0] * g.n[1]);
  return (wrapi(x + s, g.n[A]) - x) * stride;
}

// read-only loads through the non-coherent path (the kernels issue every
// load of an input before their stores to other arrays)
template <class T> __device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }
template <> __device__ __forceinline__ df ldg<df>(const df* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return df(v.x, v.y);
}

// Positive doubles order like their bit patterns: the maximum inverse
// crossing time goes through an integer atomicMax.  The block reduces in the
// compute type and converts once.
template <class T> __device__ __forceinline__ void block_max_to(T v, unsigned long long* dst) {
  __shared__ T red[BX * BY / 32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int t = threadIdx.y * BX + threadIdx.x;
  if ((t & 31) == 0) red[t >> 5] = v;
  __syncthreads();
  if (t == 0) {
    T m = red[0];
    for (int w = 1; w < BX * BY / 32; ++w) m = fmax(m, red[w]);
    const unsigned long long bits = (unsigned long long)__double_as_longlong((double)m);
    if (bits > *(volatile unsigned long long*)dst) atomicMax(dst, bits);
  }
}

// double-float values reduce as doubles
template <> __device__ __forceinline__ void block_max_to<df>(df v, unsigned long long* dst) {
  block_max_to<double>((double)v, dst);
}

// the maximum of v over the thread block, returned to every thread
// (non-negative values; a NaN is ignored)
__device__ __forceinline__ float block_max_all(float v) {
  __shared__ float red_f[BX * BY / 32];
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int t = threadIdx.y * BX + threadIdx.x;
  if ((t & 31) == 0) red_f[t >> 5] = v;
  __syncthreads();
  float m = red_f[0];
#pragma unroll
  for (int w = 1; w < BX * BY / 32; ++w) m = fmaxf(m, red_f[w]);
  return m;
}

// inverse crossing time max over l of (|v_l| + c_f,l) / d_l of one cell; the
// step is dt = C_CFL / (max over cells) (Eq. dt)
// (c_f of Eq. c_f per axis, with 1/rho and a^2 = gamma P / rho shared by the three axes)
template <class T> __device__ __forceinline__ T cell_inv_crossing(const Grid& g, const T* w8) {
  const T ir = trcp<T>(w8[0]);
  const T a2 = from_d<T>(g.gamma) * w8[4] * ir;
  const T sq[3] = {w8[5] * w8[5], w8[6] * w8[6], w8[7] * w8[7]};
  T best = T(0);
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const T t2 = (sq[(l + 1) % 3] + sq[(l + 2) % 3]) * ir;
    const T b2 = sq[l] * ir + t2;
    const T dd = a2 - b2;
    const T cf = tsqrt<T>(T(0.5) * (a2 + b2 + tsqrt<T>(dd * dd + T(4) * a2 * t2)));
    best = max_nonneg<T>(best, (fabs(w8[1 + l]) + cf) * from_d<T>(g.id[l]));
  }
  return best;
}

// primitives from a double state of one cell: rho' = max(rho, floor),
// v = m / rho', P' = max((gamma-1)(E - m.v/2 - |B_cc|^2/2), floor)
__device__ __forceinline__ PrimD prim_core_ir(const Grid& g, double rho, double ir, double m0, double m1, double m2,
                                              double e, const double* b) {
  PrimD w;
  w.b[0] = b[0];
  w.b[1] = b[1];
  w.b[2] = b[2];
  w.rho = rho;
  w.v[0] = m0 * ir;
  w.v[1] = m1 * ir;
  w.v[2] = m2 * ir;
  const double ke = 0.5 * (m0 * w.v[0] + m1 * w.v[1] + m2 * w.v[2]);
  const double me = 0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
  w.p = max_pos<double>(g.gm1 * (e - ke - me), g.p_floor);
  return w;
}

__device__ __forceinline__ PrimD prim_core(const Grid& g, double r, double m0, double m1, double m2, double e,
                                           const double* b) {
  const double rho = max_pos<double>(r, g.rho_floor);
  return prim_core_ir(g, rho, __drcp_rn(rho), m0, m1, m2, e, b);
}

// Cell-centred reference electric field E = -(v x B_cc) of one cell (Sec. 2.2
// Step 4, the reference field of the edge-field slopes), component A, from
// the stored primitives.  The kernels that write W write it beside W once per
// cell, so the edge fields read one value per cell instead of four primitives.
template <class T, int A> __device__ __forceinline__ T cell_ref(const T* w8) {
  constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
  return -(w8[1 + B] * w8[5 + C] - w8[1 + C] * w8[5 + B]);
}
template <class T> __device__ __forceinline__ void store_ref(const Fields<T, 3>& Er, int c, const T* w8) {
  if (!Er.f[0]) return;
  Er.f[0][c] = cell_ref<T, 0>(w8);
  Er.f[1][c] = cell_ref<T, 1>(w8);
  Er.f[2][c] = cell_ref<T, 2>(w8);
}

template <class T> __device__ __forceinline__ void prim_to_w8(const PrimD& p, T* w8) {
  w8[0] = from_d<T>(p.rho);
  w8[1] = from_d<T>(p.v[0]);
  w8[2] = from_d<T>(p.v[1]);
  w8[3] = from_d<T>(p.v[2]);
  w8[4] = from_d<T>(p.p);
  w8[5] = from_d<T>(p.b[0]);
  w8[6] = from_d<T>(p.b[1]);
  w8[7] = from_d<T>(p.b[2]);
}

template <class T> __device__ __forceinline__ void store_w(const Fields<T, 8>& W, int c, const PrimD& p, T* w8) {
  prim_to_w8<T>(p, w8);
#pragma unroll
  for (int f = 0; f < 8; ++f) W.f[f][c] = w8[f];
}

// x / 4 for x >= 0, exact: on the exponent bits where x is a normal double of
// exponent field >= 3 (a subtraction on the integer pipes), else (zero, tiny,
// infinite or NaN x) a multiplication, taken only in warps where a lane
// needs it
__device__ __forceinline__ double quarter_nonneg(double x) {
  const long long b = dbits(x);
  const bool fast = b >= (3LL << 52) && b < 0x7ff0000000000000LL;
  double r = __longlong_as_double(b - (2LL << 52));
  if (__any_sync(__activemask(), !fast)) {
    if (!fast) r = 0.25 * x;
  }
  return r;
}

// FP32-bulk gas-pressure recovery in double: t2 = |m|^2 / rho' + |B_cc|^2
// (twice the kinetic plus magnetic energy) and pe = E - t2 / 2, so that
// P = (gamma - 1) pe.  bsum = twice the cell-centred field (the sum of the
// two face values).  Written with explicit multiply-adds, so the forward
// step and its reverse (which repeats the floor decision) evaluate it alike;
// E - t2/2 is one fused operation (t2/2 is exact).
__device__ __forceinline__ void p_recover_f32(double ir, double m0, double m1, double m2, double e, const double* bsum,
                                              double& t2, double& pe) {
  const double mm = fma(m0, m0, fma(m1, m1, m2 * m2));
  const double bb = fma(bsum[0], bsum[0], fma(bsum[1], bsum[1], bsum[2] * bsum[2]));
  t2 = fma(mm, ir, quarter_nonneg(bb));
  pe = fma(-0.5, t2, e);
}

// FP32-bulk primitives of one cell: the gas-pressure recovery
// P = max((gamma - 1)(E - |m|^2 / (2 rho') - |B_cc|^2 / 2), P_floor) in double
// (p_recover_f32), the outputs that are stored as float (v = m / rho', B_cc)
// formed on the FP32 pipes from the rounded inputs.  Returns t2 (twice
// ke + me, for the floor reset) and pg = (gamma - 1)(E - ke - me) before the
// floor.
__device__ __forceinline__ void prim_store_f32(const Grid& g, const Fields<float, 8>& W, int c, double rho, double ir,
                                               double m0, double m1, double m2, double e, const double* bsum,
                                               float* w8, double& t2, double& pg) {
  double pe;
  p_recover_f32(ir, m0, m1, m2, e, bsum, t2, pe);
  pg = g.gm1 * pe;
  const double p = max_pos<double>(pg, g.p_floor);
  const float irf = d2f_bits(ir);
  w8[0] = d2f_bits(rho);
  w8[1] = d2f_bits(m0) * irf;
  w8[2] = d2f_bits(m1) * irf;
  w8[3] = d2f_bits(m2) * irf;
  w8[4] = d2f_bits(p);
  w8[5] = 0.5f * d2f_bits(bsum[0]);
  w8[6] = 0.5f * d2f_bits(bsum[1]);
  w8[7] = 0.5f * d2f_bits(bsum[2]);
#pragma unroll
  for (int f = 0; f < 8; ++f) W.f[f][c] = w8[f];
}

// ------------------------------------------------------------------ Step 1 --
// Primitives W of a state, and optionally (floors != nullptr) the end-of-step
// floors of the conserved state (D-12): rho < rho_floor is raised; if the
// recovered P < p_floor, E is reset so that P = p_floor.  Only the cell's own
// rho and E are written, so this is race-free in place.  The CFL maximum and
// the floor counters take interior cells only (ghost cells of a padded grid
// are copies).
template <class T>
__global__ void __launch_bounds__(BX* BY) k_prim(Grid g, Fields<double, 8> U, Fields<T, 8> W, unsigned long long* dtbits,
                                                 unsigned* flags, unsigned long long* floors, Fields<T, 3> Er) {
  const Cell p = thread_cell(g);
  T inv = T(0);
  bool wd = false;  // (double) this cell's primitives wk enter the CFL maximum
  double wk[8];
  if (p.ok) {
    const int c = p.c;
    const bool in = interior(g, p.i, p.j, p.k);
    // (rho and E are written below with the floors: plain loads; the face
    // fields are only read)
    double r = U.f[0][c], e = U.f[4][c];
    const double m0 = U.f[1][c], m1 = U.f[2][c], m2 = U.f[3][c];
    const double b0m = ldg(U.f[5] + c + p.m[0]), b0p = ldg(U.f[5] + c);
    const double b1m = ldg(U.f[6] + c + p.m[1]), b1p = ldg(U.f[6] + c);
    const double b2m = ldg(U.f[7] + c + p.m[2]), b2p = ldg(U.f[7] + c);
    // (bit-pattern tests on the integer pipes: the FP64 pipe bounds this kernel)
    if ((!pos_bits(r) || !finite_bits(e) || !finite_bits(m0) || !finite_bits(m1) || !finite_bits(m2)) && in)
      atomicOr(flags, 1u);
    if (floors && lt_pos<double>(r, g.rho_floor)) {
      r = g.rho_floor;
      U.f[0][c] = r;
      if (in) atomicAdd(&floors[0], 1ull);
    }
    const double rho = max_pos<double>(r, g.rho_floor);
    const double ir = __drcp_rn(rho);
    T w8[8];
    if constexpr (std::is_same<T, float>::value) {
      const double bs[3] = {b0m + b0p, b1m + b1p, b2m + b2p};
      double t2, pg;
      prim_store_f32(g, W, c, rho, ir, m0, m1, m2, e, bs, w8, t2, pg);
      store_ref<T>(Er, c, w8);
      if (floors && lt_pos<double>(pg, g.p_floor)) {
        U.f[4][c] = g.p_floor * g.igm1 + 0.5 * t2;
        if (in) atomicAdd(&floors[1], 1ull);
      }
      if (dtbits && in) inv = cell_inv_crossing<T>(g, w8);
    } else {
      double b[3];
      b[0] = 0.5 * (b0m + b0p);
      b[1] = 0.5 * (b1m + b1p);
      b[2] = 0.5 * (b2m + b2p);
      if (floors) {
        const double ke = 0.5 * (m0 * (m0 * ir) + m1 * (m1 * ir) + m2 * (m2 * ir));
        const double me = 0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        if (lt_pos<double>(g.gm1 * (e - ke - me), g.p_floor)) {
          e = g.p_floor * g.igm1 + ke + me;
          U.f[4][c] = e;
          if (in) atomicAdd(&floors[1], 1ull);
        }
      }
      const PrimD pw = prim_core_ir(g, rho, ir, m0, m1, m2, e, b);
      store_w<T>(W, c, pw, w8);
      store_ref<T>(Er, c, w8);
      if constexpr (std::is_same<T, double>::value) {
        if (dtbits && in) {
          wd = true;
#pragma unroll
          for (int f = 0; f < 8; ++f) wk[f] = w8[f];
        }
      } else {
        if (dtbits && in) inv = cell_inv_crossing<T>(g, w8);
      }
    }
  }
  if constexpr (std::is_same<T, double>::value) {
    // The CFL maximum of the FP64 step.  Each interior cell's rate is first
    // estimated in float from its primitives rounded to float.  Where the
    // grid's 1/d_l and the cell's density and pressure lie in [1e-9, 1e9],
    // every intermediate of the estimate is a normal float, an overflow
    // (giving a non-finite estimate) or an underflow whose absolute error
    // is negligible against a^2 = gamma P / rho, so a finite estimate is
    // within a relative 1e-5 of the exact rate.  The block maximum M of
    // those estimates then bounds their cells' exact rates, and only a cell
    // whose estimate reaches M (1 - 1e-4), or whose estimate is not trusted
    // (outside the range, not finite), can hold the block's exact maximum.
    // Those cells evaluate the double rate: the block's maximum is that of
    // the per-cell double evaluation, bit for bit, at a fraction of the FP64
    // work (typically one warp in a few per block).
    if (dtbits) {
      auto in_range = [](double x) {  // 1e-9 <= x <= 1e9, on the bit pattern (integer pipes)
        const long long b = dbits(x);
        return b >= dbits(1e-9) && b <= dbits(1e9);
      };
      const bool grid_ok = in_range(g.id[0]) && in_range(g.id[1]) && in_range(g.id[2]);
      float est = 0.0f;
      bool trusted = false;
      if (wd && grid_ok && in_range(wk[0]) && in_range(wk[4])) {
        float wf[8];
#pragma unroll
        for (int f = 0; f < 8; ++f) wf[f] = d2f_bits(wk[f]);
        est = cell_inv_crossing<float>(g, wf);
        trusted = est <= 3.402823466e38f;  // false for an infinity or a NaN
      }
      const float m = block_max_all(trusted ? est : 0.0f);
      const bool cand = wd && (!trusted || !(est < m * (1.0f - 1e-4f)));
      double inv_d = 0.0;
      if (cand) inv_d = cell_inv_crossing<double>(g, wk);
      block_max_to<double>(inv_d, dtbits);
    }
  } else {
    if (dtbits) block_max_to<T>(inv, dtbits);
  }
}

// directional 7-vector (rho, v_n, v_t1, v_t2, P, B_t1, B_t2) of cell q
template <int A, class T> __device__ __forceinline__ void load_dir(const T* __restrict__ W, long long N, long long q, T* w) {
  constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
  w[0] = W[q];
  w[1] = W[(1 + A) * N + q];
  w[2] = W[(1 + B) * N + q];
  w[3] = W[(1 + C) * N + q];
  w[4] = W[4 * N + q];
  w[5] = W[(5 + B) * N + q];
  w[6] = W[(5 + C) * N + q];
}
template <int A, class T> __device__ __forceinline__ void load_dir(const Fields<const T, 8>& W, int q, T* w) {
  constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
  w[0] = ldg(W.f[0] + q);
  w[1] = ldg(W.f[1 + A] + q);
  w[2] = ldg(W.f[1 + B] + q);
  w[3] = ldg(W.f[1 + C] + q);
  w[4] = ldg(W.f[4] + q);
  w[5] = ldg(W.f[5 + B] + q);
  w[6] = ldg(W.f[5 + C] + q);
}

// -------------------------------------------------------------- Steps 2-3 --
// one axis per launch: a thread solving three Riemann problems in sequence
// holds too many registers for the occupancy the double-float arithmetic
// needs to hide its latencies.  BA: the face field B_A of the state.
template <class T, int A>
__global__ void __launch_bounds__(BX* BY) k_flux_pcm(Grid g, Fields<const T, 8> W, const double* __restrict__ BA,
                                                     Fields<T, 7> FA) {
  const Cell p = thread_cell(g);
  if (!p.ok) return;
  const int c = p.c;
  T wl[7], wr[7], f[7];
  load_dir<A>(W, c, wl);
  load_dir<A>(W, c + p.p[A], wr);
  hlld<T>(from_d<T>(g.gamma), from_d<T>(g.igm1), wl, wr, from_d<T>(ldg(BA + c)), f);
#pragma unroll
  for (int q = 0; q < 7; ++q) FA.f[q][c] = f[q];
}

// ------------------------------------------------------------------ Step 6 --
template <class T> __device__ __forceinline__ void floor_face(const Grid& g, T* w) {
  w[0] = max_pos<T>(w[0], from_d<T>(g.rho_floor));
  w[4] = max_pos<T>(w[4], from_d<T>(g.p_floor));
}

// blocks of 128 threads per SM requested from the register allocator (4:
// at most 128 registers per thread).  The double and double-float PPMC and
// the double PLMC kernels fit 128 registers without spilling; the
// double-float PLMC kernel spills 40 bytes there and still runs 9 % faster
// than at 3 blocks (168 registers, no spill): its dependent float-pair
// chains need the extra warps.  (The double-float flux kernels, 112-119
// registers, lose 2 % at 5 blocks with 40-68 bytes of spill; the double PLMC
// kernel, 108 registers, loses 5 % at 5 blocks, 96 registers.)
template <class T, int RECON> struct ReconMinBlocks { static constexpr int v = 4; };

// interface states of cell p along A (Step 6): wl = W_{L,i+1/2} (the cell's
// state at its upper face), wr = W_{R,i-1/2} (at its lower face), floored
template <class T, int RECON, int A>
__device__ __forceinline__ void recon_cell(const Grid& g, const Fields<const T, 8>& W, const Cell& p, T* wl, T* wr) {
  const int c = p.c;
  const T bn = ldg(W.f[5 + A] + c);
  if (RECON == 0) {
    load_dir<A>(W, c, wl);
#pragma unroll
    for (int q = 0; q < 7; ++q) wr[q] = wl[q];
  } else if (RECON == 1 || RECON == 3) {
    T wm[7], w0[7], wp[7];
    load_dir<A>(W, c + p.m[A], wm);
    load_dir<A>(W, c, w0);
    load_dir<A>(W, c + p.p[A], wp);
    if (RECON == 1) plmc<T>(from_d<T>(g.gamma), wm, w0, wp, bn, wl, wr);
    else plm_prim<T>(wm, w0, wp, wl, wr);
  } else {
    T w[5][7];
#pragma unroll
    for (int s = -2; s <= 2; ++s) load_dir<A>(W, c + off<A>(g, p, s), w[s + 2]);
    ppmc<T>(from_d<T>(g.gamma), w, bn, wl, wr);
  }
  floor_face<T>(g, wl);
  floor_face<T>(g, wr);
}

template <class T, int RECON, int A>
__global__ void __launch_bounds__(BX* BY, ReconMinBlocks<T, RECON>::v) k_recon(Grid g, Fields<const T, 8> W,
                                                                             Fields<T, 7> WL, Fields<T, 7> WR) {
  const Cell p = thread_cell(g);
  if (!p.ok) return;
  T wl[7], wr[7];
  recon_cell<T, RECON, A>(g, W, p, wl, wr);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    WL.f[q][p.c] = wl[q];
    WR.f[q][p.c] = wr[q];
  }
}

// ------------------------------------------------------------------ Step 7 --
// BfA: the half-step face field B_A
template <class T, int A>
__global__ void __launch_bounds__(BX* BY) k_flux_hlld(Grid g, Fields<const T, 7> WL, Fields<const T, 7> WR,
                                                      const T* __restrict__ BfA, Fields<T, 7> FA) {
  const Cell p = thread_cell(g);
  if (!p.ok) return;
  const int c = p.c, cn = c + p.p[A];
  T wl[7], wr[7], f[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    wl[q] = ldg(WL.f[q] + c);
    wr[q] = ldg(WR.f[q] + cn);
  }
  hlld<T>(from_d<T>(g.gamma), from_d<T>(g.igm1), wl, wr, ldg(BfA + c), f);
#pragma unroll
  for (int q = 0; q < 7; ++q) FA.f[q][c] = f[q];
}

// The float Riemann kernel keeps restrict-qualified base pointers with
// 64-bit indices: measured at 512^3 (PPMC turbulent box), 6.25 ms per step
// for its three launches against 6.89 ms in the pointer-table form above;
// the double and float-pair Riemann kernels are as fast or faster in the
// table form.
template <class T, int A>
__global__ void __launch_bounds__(BX* BY) k_flux_hlld_r(Grid g, const T* __restrict__ WL, const T* __restrict__ WR,
                                                        const T* __restrict__ Bf, T* __restrict__ F) {
  const CellIdx ci = cell_of_thread(g);
  if (!ci.ok) return;
  const long long N = g.N, c = cidx(g, ci.i, ci.j, ci.k), cn = nb<A>(g, ci.i, ci.j, ci.k, 1);
  T wl[7], wr[7], f[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    wl[q] = WL[q * N + c];
    wr[q] = WR[q * N + cn];
  }
  hlld<T>(from_d<T>(g.gamma), from_d<T>(g.igm1), wl, wr, Bf[A * N + c], f);
#pragma unroll
  for (int q = 0; q < 7; ++q) F[((long long)A * 7 + q) * N + c] = f[q];
}

// ------------------------------------------------------------ Steps 4, 8 --
// Edge A of cell p at p + e_B/2 + e_C/2, (B, C) = (A+1, A+2): mean of the four
// face fields plus the upwinded "face minus reference" slopes (Eq. emf-edge,
// Eqs. emf-upwind-slope, emf-slope), upwinded by the sign of the mass flux of
// the face the slope sits on (mean when it is exactly zero).
// The slope upwinded by the mass flux m: (f_lo - r_lo) where m > 0, (f_hi -
// r_hi) where m < 0, their mean where m == 0.
template <class T> __device__ __forceinline__ T upwind(T m, T flo, T rlo, T fhi, T rhi) {
  const T lo = flo - rlo, hi = fhi - rhi;
  return m > T(0) ? lo : (m < T(0) ? hi : T(0.5) * (lo + hi));
}
// double: the sign tests on the bit pattern (integer pipes); the operands are
// selected first, so one difference is formed per slope, and the mean
// (needed only for an exactly zero mass flux, e.g. a fluid at rest) is a
// call made only in warps where some lane needs it -- inlined, the compiler
// evaluates it in every warp, two FP64-pipe instructions per slope
__device__ __noinline__ static double upwind_mean(double flo, double rlo, double fhi, double rhi) {
  return 0.5 * ((flo - rlo) + (fhi - rhi));
}
template <> __device__ __forceinline__ double upwind<double>(double m, double flo, double rlo, double fhi, double rhi) {
  const long long b = dbits(m);
  const bool z = (b & kAbsBits) == 0;
  const bool lo = b > 0;
  double d = (lo ? flo : fhi) - (lo ? rlo : rhi);
  if (__any_sync(__activemask(), z)) {
    if (z) d = upwind_mean(flo, rlo, fhi, rhi);
  }
  return d;
}

template <class T, int A, bool REF>
__device__ __forceinline__ T edge_field(const Grid& g, const Fields<const T, 8>& W, const Fields<const T, 21>& F,
                                        const Fields<const T, 3>& Er, const Cell& p) {
  constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
  const int q00 = p.c, qb = q00 + p.p[B], qc = q00 + p.p[C], qbc = qb + p.p[C];
  const T* Fbm = F.f[B * 7];      // mass flux of axis B
  const T* Fbb = F.f[B * 7 + 5];  // B-field flux 5 of axis B
  const T* Fcm = F.f[C * 7];
  const T* Fcb = F.f[C * 7 + 6];
  auto ref = [&](int q) {
    if constexpr (REF) {
      return ldg(Er.f[A] + q);
    } else {
      const T w8[8] = {T(0), ldg(W.f[1] + q), ldg(W.f[2] + q), ldg(W.f[3] + q),
                       T(0), ldg(W.f[5] + q), ldg(W.f[6] + q), ldg(W.f[7] + q)};
      return cell_ref<T, A>(w8);
    }
  };
  const T bf0 = -ldg(Fbb + q00), bfc = -ldg(Fbb + qc);
  const T cf0 = ldg(Fcb + q00), cfb = ldg(Fcb + qb);
  const T r00 = ref(q00), rb = ref(qb), rc = ref(qc), rbc = ref(qbc);
  const T avg = T(0.25) * (bfc + bf0 + cfb + cf0);
  const T Dcp = upwind<T>(ldg(Fbm + qc), cf0, rc, cfb, rbc);
  const T Dcm = upwind<T>(ldg(Fbm + q00), cf0, r00, cfb, rb);
  const T Dbp = upwind<T>(ldg(Fcm + qb), bf0, rb, bfc, rbc);
  const T Dbm = upwind<T>(ldg(Fcm + q00), bf0, r00, bfc, rc);
  return avg + T(0.25) * (Dcp + Dcm + Dbp + Dbm);
}

// REF: the cells' reference fields come from Er (written with W), else from W
template <class T, bool REF>
__global__ void __launch_bounds__(BX* BY) k_emf(Grid g, Fields<const T, 8> W, Fields<const T, 21> F,
                                                Fields<const T, 3> Er, Fields<T, 3> E) {
  const Cell p = thread_cell(g);
  if (!p.ok) return;
  const T e0 = edge_field<T, 0, REF>(g, W, F, Er, p);
  const T e1 = edge_field<T, 1, REF>(g, W, F, Er, p);
  const T e2 = edge_field<T, 2, REF>(g, W, F, Er, p);
  E.f[0][p.c] = e0;
  E.f[1][p.c] = e1;
  E.f[2][p.c] = e2;
}

// The edge fields of the FP64 step keep the addressing of restrict-qualified
// base pointers with 64-bit indices: measured at 512^3 (PPMC turbulent box),
// this form takes 24.4 ms per step against 36.6 ms for the pointer-table form
// above (same registers, no spill), while the float and double-float edge
// kernels are faster in the table form (3.2 against 4.8 ms, 7.8 against
// 8.9 ms).
template <class T, int A, bool REF>
__device__ __forceinline__ T edge_field_r(const Grid& g, const T* __restrict__ W, const T* __restrict__ F,
                                          const T* __restrict__ Er, int i, int j, int k) {
  constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
  const long long N = g.N;
  int pb[3] = {i, j, k}, pc[3] = {i, j, k}, pbc[3] = {i, j, k};
  pb[B] = wrapi(pb[B] + 1, g.n[B]);
  pc[C] = wrapi(pc[C] + 1, g.n[C]);
  pbc[B] = pb[B];
  pbc[C] = pc[C];
  const long long q00 = cidx(g, i, j, k), qb = cidx(g, pb[0], pb[1], pb[2]);
  const long long qc = cidx(g, pc[0], pc[1], pc[2]), qbc = cidx(g, pbc[0], pbc[1], pbc[2]);
  const T* Fb = F + (long long)B * 7 * N;
  const T* Fc = F + (long long)C * 7 * N;
  auto ref = [&](long long q) {
    if constexpr (REF) {
      return Er[(long long)A * N + q];
    } else {
      const T w8[8] = {T(0), W[N + q], W[2 * N + q], W[3 * N + q], T(0), W[5 * N + q], W[6 * N + q], W[7 * N + q]};
      return cell_ref<T, A>(w8);
    }
  };
  const T bf0 = -Fb[5 * N + q00], bfc = -Fb[5 * N + qc];
  const T cf0 = Fc[6 * N + q00], cfb = Fc[6 * N + qb];
  const T r00 = ref(q00), rb = ref(qb), rc = ref(qc), rbc = ref(qbc);
  const T avg = T(0.25) * (bfc + bf0 + cfb + cf0);
  const T Dcp = upwind<T>(Fb[qc], cf0, rc, cfb, rbc);
  const T Dcm = upwind<T>(Fb[q00], cf0, r00, cfb, rb);
  const T Dbp = upwind<T>(Fc[qb], bf0, rb, bfc, rbc);
  const T Dbm = upwind<T>(Fc[q00], bf0, r00, bfc, rc);
  return avg + T(0.25) * (Dcp + Dcm + Dbp + Dbm);
}

template <class T, bool REF>
__global__ void __launch_bounds__(BX* BY) k_emf_r(Grid g, const T* __restrict__ W, const T* __restrict__ F,
                                                  const T* __restrict__ Er, T* __restrict__ E) {
  const CellIdx ci = cell_of_thread(g);
  if (!ci.ok) return;
  const long long N = g.N, c = cidx(g, ci.i, ci.j, ci.k);
  E[c] = edge_field_r<T, 0, REF>(g, W, F, Er, ci.i, ci.j, ci.k);
  E[N + c] = edge_field_r<T, 1, REF>(g, W, F, Er, ci.i, ci.j, ci.k);
  E[2 * N + c] = edge_field_r<T, 2, REF>(g, W, F, Er, ci.i, ci.j, ci.k);
}

// ------------------------------------------------------------ Steps 5, 9 --
// solver-frame component of the global field f (0 rho, 1-3 m, 4 E) in the flux of axis a
__device__ __forceinline__ int comp_of(int f, int a) {
  return (f == 0 || f == 4) ? f : 1 + ((f - 1 - a + 3) % 3);
}

// curl term of face A of cell q: (E_C(q) - E_C(q - e_B))/d_B - (E_B(q) -
// E_B(q - e_C))/d_C; oB, oC: the offsets from q to q - e_B and q - e_C.
// EXACT: each edge difference is exact (float edges: as a float pair by
// TwoSum; double edges: widened before differencing), so the discrete
// divergence of the update telescopes to double round-off whatever the
// compute type (the FP32-bulk full update keeps div B at FP64 round-off).
template <class T, bool EXACT, int A>
__device__ __forceinline__ double face_curl(const Grid& g, const Fields<const T, 3>& E, int q, int oB, int oC) {
  constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
  const T* EB = E.f[B];
  const T* EC = E.f[C];
  if constexpr (EXACT && std::is_same<T, float>::value) {
    const df dc = two_sum(ldg(EC + q), -ldg(EC + q + oB));
    const df db = two_sum(ldg(EB + q), -ldg(EB + q + oC));
    return (double)(dc * df(g.id[B]) - db * df(g.id[C]));
  } else if (EXACT) {
    return (to_d<T>(ldg(EC + q)) - to_d<T>(ldg(EC + q + oB))) * g.id[B] -
           (to_d<T>(ldg(EB + q)) - to_d<T>(ldg(EB + q + oC))) * g.id[C];
  }
  return to_d<T>((ldg(EC + q) - ldg(EC + q + oB)) * from_d<T>(g.id[B]) -
                 (ldg(EB + q) - ldg(EB + q + oC)) * from_d<T>(g.id[C]));
}

template <bool NC> __device__ __forceinline__ double ldu(const double* p) {
  if constexpr (NC) return ldg(p);
  else return *p;
}

// the factor (dt or dt / 2) / d_a of axis a in the compute type, from the
// step scalars (formed once per step by the dt kernels)
template <class T, bool HALF> __device__ __forceinline__ T step_factor(const StepScalars& S, int a) {
  if constexpr (std::is_same<T, float>::value) {
    return HALF ? S.hd_half_f[a] : d2f_bits(S.hd_full[a]);
  } else if constexpr (std::is_same<T, df>::value) {
    return HALF ? df(S.hd_half_hi[a], S.hd_half_lo[a]) : df(S.hd_full_hi[a], S.hd_full_lo[a]);
  } else {
    return HALF ? S.hd_half[a] : S.hd_full[a];
  }
}

// new hydro state of one cell: U0 - h sum_a (F_a(p) - F_a(p - e_a)) / d_a,
// with h / d_a from the step scalars (HALF: h = dt / 2).  EXACT: every flux
// difference is exact -- in double for double fluxes, as a float pair
// (TwoSum, FP32 pipes) for float fluxes -- and the increment is accumulated
// in double or float pairs, so sums over the periodic box telescope to
// round-off: the FP32-bulk full update conserves rho, m, E at the FP64 level.
// Otherwise (FP32-bulk and double-float half step) the increment is formed
// in T and added to the double state.  NC: U0 is read-only in the kernel
// (non-coherent loads).
template <class T, bool EXACT, bool NC, bool HALF>
__device__ __forceinline__ void hydro_update(const Fields<const double, 8>& U0, const Fields<const T, 21>& F,
                                             const StepScalars& S, const Cell& p, double* out5) {
  const int c = p.c;
  const double* hd = HALF ? S.hd_half : S.hd_full;
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    if constexpr (EXACT && std::is_same<T, float>::value) {
      df inc(0.0f, 0.0f);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T* Fa = F.f[a * 7 + comp_of(f, a)];
        const df hdf = HALF ? df(S.hd_half_hi[a], S.hd_half_lo[a]) : df(S.hd_full_hi[a], S.hd_full_lo[a]);
        inc += hdf * two_sum(ldg(Fa + c), -ldg(Fa + c + p.m[a]));
      }
      out5[f] = ldu<NC>(U0.f[f] + c) - (double)inc;
    } else if (EXACT) {
      double acc = ldu<NC>(U0.f[f] + c);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T* Fa = F.f[a * 7 + comp_of(f, a)];
        acc -= hd[a] * (to_d<T>(ldg(Fa + c)) - to_d<T>(ldg(Fa + c + p.m[a])));
      }
      out5[f] = acc;
    } else {
      T inc = T(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T* Fa = F.f[a * 7 + comp_of(f, a)];
        inc -= step_factor<T, HALF>(S, a) * (ldg(Fa + c) - ldg(Fa + c + p.m[a]));
      }
      out5[f] = ldu<NC>(U0.f[f] + c) + to_d<T>(inc);
    }
  }
}

// new upper face B_A of cell q: B0 - h curl
template <class T, bool EXACT, bool NC, int A>
__device__ __forceinline__ double face_update(const Grid& g, const Fields<const double, 8>& U0,
                                              const Fields<const T, 3>& E, double h, int q, int oB, int oC) {
  const double cu = face_curl<T, EXACT, A>(g, E, q, oB, oC);
  return ldu<NC>(U0.f[5 + A] + q) - h * cu;
}

template <class T, int K> __device__ __forceinline__ Fields<const T, K> as_const(const Fields<T, K>& a) {
  Fields<const T, K> r;
#pragma unroll
  for (int q = 0; q < K; ++q) r.f[q] = a.f[q];
  return r;
}

// Step 5: W^{n+1/2} (from U^{n+1/2}) and the half-step faces; h = dt/2 (D-1).
// dtp: the StepScalars of the step.
template <class T>
__global__ void __launch_bounds__(BX* BY) k_update_half(Grid g, Fields<const double, 8> U0, Fields<const T, 21> F,
                                                        Fields<const T, 3> E, const double* __restrict__ dtp,
                                                        Fields<T, 8> W, Fields<T, 3> Bh, unsigned* flags,
                                                        Fields<T, 3> Er) {
  const Cell p = thread_cell(g);
  if (!p.ok) return;
  const int c = p.c;
  const StepScalars& S = *reinterpret_cast<const StepScalars*>(dtp);
  const double h = S.h_half;
  // FP64: double differences; FP32-bulk and df half step: increments in T
  constexpr bool X = sizeof(T) == 8 && Exact<T>::full;
  double u5[5];
  hydro_update<T, X, true, true>(U0, F, S, p, u5);
  // the cell's upper faces and its lower faces (the upper faces of p - e_a)
  const double bx = face_update<T, X, true, 0>(g, U0, E, h, c, p.m[1], p.m[2]);
  const double by = face_update<T, X, true, 1>(g, U0, E, h, c, p.m[2], p.m[0]);
  const double bz = face_update<T, X, true, 2>(g, U0, E, h, c, p.m[0], p.m[1]);
  const double bxm = face_update<T, X, true, 0>(g, U0, E, h, c + p.m[0], p.m[1], p.m[2]);
  const double bym = face_update<T, X, true, 1>(g, U0, E, h, c + p.m[1], p.m[2], p.m[0]);
  const double bzm = face_update<T, X, true, 2>(g, U0, E, h, c + p.m[2], p.m[0], p.m[1]);
  Bh.f[0][c] = from_d<T>(bx);
  Bh.f[1][c] = from_d<T>(by);
  Bh.f[2][c] = from_d<T>(bz);
  // (the outer ghost layers of a padded grid see the wrap and carry no check)
  if ((!pos_bits(u5[0]) || !finite_bits(u5[4])) && interior(g, p.i, p.j, p.k)) atomicOr(flags, 1u);
  T w8[8];
  if constexpr (std::is_same<T, float>::value) {
    const double bs[3] = {bxm + bx, bym + by, bzm + bz};
    const double rho = max_pos<double>(u5[0], g.rho_floor);
    double t2, pg;
    prim_store_f32(g, W, c, rho, __drcp_rn(rho), u5[1], u5[2], u5[3], u5[4], bs, w8, t2, pg);
  } else {
    const double bcc[3] = {0.5 * (bxm + bx), 0.5 * (bym + by), 0.5 * (bzm + bz)};
    const PrimD pw = prim_core(g, u5[0], u5[1], u5[2], u5[3], u5[4], bcc);
    store_w<T>(W, c, pw, w8);
  }
  store_ref<T>(Er, c, w8);
}

// Step 9: U^{n+1} in place.  Each thread reads and writes only its own cell of
// U (hydro fields and its three upper faces), so the update is race-free in
// place; floors, W^{n+1} and the next dt follow in k_prim with floors on.
template <class T>
__global__ void __launch_bounds__(BX* BY) k_update_full(Grid g, Fields<double, 8> U, Fields<const T, 21> F,
                                                        Fields<const T, 3> E, const double* __restrict__ dtp) {
  const Cell p = thread_cell(g);
  if (!p.ok) return;
  const int c = p.c;
  const StepScalars& S = *reinterpret_cast<const StepScalars*>(dtp);
  const double h = S.dt;
  const Fields<const double, 8> Uc = as_const(U);
  double u5[5];
  constexpr bool X = Exact<T>::full;
  hydro_update<T, X, false, false>(Uc, F, S, p, u5);
  const double bx = face_update<T, X, false, 0>(g, Uc, E, h, c, p.m[1], p.m[2]);
  const double by = face_update<T, X, false, 1>(g, Uc, E, h, c, p.m[2], p.m[0]);
  const double bz = face_update<T, X, false, 2>(g, Uc, E, h, c, p.m[0], p.m[1]);
#pragma unroll
  for (int f = 0; f < 5; ++f) U.f[f][c] = u5[f];
  U.f[5][c] = bx;
  U.f[6][c] = by;
  U.f[7][c] = bz;
}

template <class T> __global__ void k_widen(const T* __restrict__ src, double* __restrict__ dst, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    dst[q] = (double)src[q];
}

template <class T> __global__ void k_narrow(const double* __restrict__ src, T* __restrict__ dst, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
    dst[q] = (T)src[q];
}

// the step scalars of step size dt (the factors formed exactly as the
// update kernels would form them: (dt / 2) / d_a = (0.5 dt) id_a)
__device__ __forceinline__ void set_step_scalars(const Grid& g, StepScalars* S, double dt) {
  S->dt = dt;
  S->h_half = 0.5 * dt;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    S->hd_full[a] = dt * g.id[a];
    S->hd_half[a] = S->h_half * g.id[a];
    S->hd_half_f[a] = d2f_bits(S->hd_half[a]);
    const df x(S->hd_full[a]), y(S->hd_half[a]);
    S->hd_full_hi[a] = x.hi;
    S->hd_full_lo[a] = x.lo;
    S->hd_half_hi[a] = y.hi;
    S->hd_half_lo[a] = y.lo;
  }
}

#ifdef MHD_SCALAR_KERNELS
// --------------------------------------------------------- small kernels --
__global__ void k_set_dt(Grid g, double* dt_cur, double value) {
  set_step_scalars(g, reinterpret_cast<StepScalars*>(dt_cur), value);
}

// dt = cfl / max inverse crossing time; records it and re-arms the reduction word
// dt = C_CFL / max rate (Eq. dt), shortened to t_end - t when it would step
// past t_end (t_end = +inf: no end time); the shortened step lands on t_end.
__global__ void k_finish_dt(Grid g, unsigned long long* dtbits, double* dt_cur, double* dt_log, int s,
                            unsigned* flags, double t_end) {
  const double m = __longlong_as_double((long long)dtbits[0]);
  double dt = g.cfl / m;
  if (!(dt > 0.0) || !isfinite(dt)) atomicOr(flags, 2u);
  const double t = dt_cur[1];  // simulated time of the current run
  if (dt >= t_end - t) {
    dt = t_end - t;
    dt_cur[1] = t_end;
  } else {
    dt_cur[1] = t + dt;
  }
  set_step_scalars(g, reinterpret_cast<StepScalars*>(dt_cur), dt);
  if (dt_log) dt_log[s] = dt;
  dtbits[0] = 0ull;  // +0.0
}

// ------------------------------------------------- outflow ghost cells --
// Up (grid gp) holds the caller's grid in its interior box [lo, hi); Ui is
// the caller's state (grid gi).  dir = 0: Ui -> Up; dir = 1: Up -> Ui.
__global__ void k_pad_copy(Grid gp, Grid gi, double* Up, double* Ui, int dir) {
  const long long Ni = gi.N;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 8 * Ni;
       q += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(q / Ni);
    const long long c = q - f * Ni;
    const int i = (int)(c % gi.n[0]), j = (int)((c / gi.n[0]) % gi.n[1]);
    const int k = (int)(c / ((long long)gi.n[0] * gi.n[1]));
    const long long cp = f * gp.N + cidx(gp, i + gp.lo[0], j + gp.lo[1], k + gp.lo[2]);
    if (dir == 0) Up[cp] = Ui[q];
    else Ui[q] = Up[cp];
  }
}

// Subdomain of a periodic global grid (gg): every cell of the padded
// subdomain state Up (grid gp, interior box [lo, hi)) takes the global cell
// at offset off + (p - lo), wrapped periodically: interior and halo in one
// gather.
__global__ void k_gather_sub(Grid gp, Grid gg, int o0, int o1, int o2, const double* __restrict__ Ug,
                             double* __restrict__ Up) {
  const long long N = gp.N;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % gp.n[0]), j = (int)((c / gp.n[0]) % gp.n[1]);
    const int k = (int)(c / ((long long)gp.n[0] * gp.n[1]));
    int gi = (o0 + i - gp.lo[0]) % gg.n[0], gj = (o1 + j - gp.lo[1]) % gg.n[1], gk = (o2 + k - gp.lo[2]) % gg.n[2];
    gi += gi < 0 ? gg.n[0] : 0;
    gj += gj < 0 ? gg.n[1] : 0;
    gk += gk < 0 ? gg.n[2] : 0;
    const long long s = cidx(gg, gi, gj, gk);
#pragma unroll
    for (int f = 0; f < 8; ++f) Up[f * N + c] = Ug[f * gg.N + s];
  }
}

// the interior box of Up into the global state at offset off (no wrap: the
// subdomain lies inside the global grid)
__global__ void k_scatter_sub(Grid gp, Grid gg, int o0, int o1, int o2, const double* __restrict__ Up,
                              double* __restrict__ Ug) {
  const int ni = gp.hi[0] - gp.lo[0], nj = gp.hi[1] - gp.lo[1], nk = gp.hi[2] - gp.lo[2];
  const long long M = (long long)ni * nj * nk;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < 8 * M; q += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(q / M);
    const long long c = q - f * M;
    const int i = (int)(c % ni), j = (int)((c / ni) % nj), k = (int)(c / ((long long)ni * nj));
    Ug[f * gg.N + cidx(gg, o0 + i, o1 + j, o2 + k)] = Up[f * gp.N + cidx(gp, gp.lo[0] + i, gp.lo[1] + j, gp.lo[2] + k)];
  }
}

// every cell of Up outside the interior box takes all 8 fields (face fields
// included) of the nearest interior cell: zero-gradient (outflow) ghosts
__global__ void k_fill_ghosts(Grid gp, double* Up) {
  const long long N = gp.N;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(c % gp.n[0]), j = (int)((c / gp.n[0]) % gp.n[1]);
    const int k = (int)(c / ((long long)gp.n[0] * gp.n[1]));
    if (interior(gp, i, j, k)) continue;
    const int si = min(max(i, gp.lo[0]), gp.hi[0] - 1);
    const int sj = min(max(j, gp.lo[1]), gp.hi[1] - 1);
    const int sk = min(max(k, gp.lo[2]), gp.hi[2] - 1);
    const long long s = cidx(gp, si, sj, sk);
#pragma unroll
    for (int f = 0; f < 8; ++f) Up[f * N + c] = Up[f * N + s];
  }
}

// ------------------------------------------------------------ diagnostics --
// Per-block partial sums of the 8 fields and max |div B| over 1024 cells, then
// one block combines the partials in a fixed order: deterministic results.
// The sums are compensated: every partial carries the rounding error of its
// additions (TwoSum, Knuth) beside its value and the two are added at the end
// (pairwise summation with Neumaier-style error carrying), so the totals are
// accurate to about one rounding of the result whatever the cell count.
constexpr int DIAG_T = 1024;
static_assert(DIAG_T == kDiagCells, "one partial block of the diagnostics reduces kDiagCells cells");

__device__ __forceinline__ void diag_add(double& s, double& c, double s2, double c2) {
  const double t = s + s2;
  const double v = t - s;
  c += (s - (t - v)) + (s2 - v) + c2;
  s = t;
}

// red layout: [9][nblk] partial values (sums of fields 0-7, max |div B|), then
// [8][nblk] the compensations of the 8 sums
__global__ void __launch_bounds__(DIAG_T) k_diag_partial(Grid g, const double* __restrict__ U, double* red, int nblk) {
  __shared__ double sh[DIAG_T / 32][9];
  __shared__ double shc[DIAG_T / 32][8];
  const long long N = g.N;
  const long long c = (long long)blockIdx.x * DIAG_T + threadIdx.x;
  double v[9], e[8];
#pragma unroll
  for (int f = 0; f < 9; ++f) v[f] = 0.0;
#pragma unroll
  for (int f = 0; f < 8; ++f) e[f] = 0.0;
  if (c < N) {
    const int i = (int)(c % g.n[0]);
    const int j = (int)((c / g.n[0]) % g.n[1]);
    const int k = (int)(c / ((long long)g.n[0] * g.n[1]));
#pragma unroll
    for (int f = 0; f < 8; ++f) v[f] = U[f * N + c];
    // lower faces; on an outflow axis the first cell's lower face is its ghost
    // copy, equal to the cell's own upper face
    const long long lx = (g.bc[0] && i == 0) ? c : nb<0>(g, i, j, k, -1);
    const long long ly = (g.bc[1] && j == 0) ? c : nb<1>(g, i, j, k, -1);
    const long long lz = (g.bc[2] && k == 0) ? c : nb<2>(g, i, j, k, -1);
    const double dv = (U[5 * N + c] - U[5 * N + lx]) * g.id[0] + (U[6 * N + c] - U[6 * N + ly]) * g.id[1] +
                      (U[7 * N + c] - U[7 * N + lz]) * g.id[2];
    v[8] = fabs(dv);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      const double s2 = __shfl_xor_sync(0xffffffffu, v[f], o), c2 = __shfl_xor_sync(0xffffffffu, e[f], o);
      diag_add(v[f], e[f], s2, c2);
    }
    v[8] = fmax(v[8], __shfl_xor_sync(0xffffffffu, v[8], o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int f = 0; f < 9; ++f) sh[w][f] = v[f];
#pragma unroll
    for (int f = 0; f < 8; ++f) shc[w][f] = e[f];
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    const int f = threadIdx.x;
    double a = sh[0][f], ac = f < 8 ? shc[0][f] : 0.0;
    for (int q = 1; q < DIAG_T / 32; ++q) {
      if (f == 8)
        a = fmax(a, sh[q][f]);
      else
        diag_add(a, ac, sh[q][f], shc[q][f]);
    }
    red[(long long)f * nblk + blockIdx.x] = a;
    if (f < 8) red[(long long)(9 + f) * nblk + blockIdx.x] = ac;
  }
}

__global__ void __launch_bounds__(DIAG_T) k_diag_final(const double* red_in, double* out, int nblk) {
  __shared__ double sh[DIAG_T], shc[DIAG_T];
  for (int f = 0; f < 9; ++f) {
    double a = 0.0, ac = 0.0;
    for (int q = threadIdx.x; q < nblk; q += DIAG_T) {
      const double x = red_in[(long long)f * nblk + q];
      if (f == 8)
        a = fmax(a, x);
      else
        diag_add(a, ac, x, red_in[(long long)(9 + f) * nblk + q]);
    }
    sh[threadIdx.x] = a;
    shc[threadIdx.x] = ac;
    __syncthreads();
    for (int o = DIAG_T / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        if (f == 8) {
          sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        } else {
          double s1 = sh[threadIdx.x], c1 = shc[threadIdx.x];
          diag_add(s1, c1, sh[threadIdx.x + o], shc[threadIdx.x + o]);
          sh[threadIdx.x] = s1;
          shc[threadIdx.x] = c1;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) out[f] = f == 8 ? sh[0] : sh[0] + shc[0];
    __syncthreads();
  }
}

#endif  // MHD_SCALAR_KERNELS

// --------------------------------------------------------------- launchers --

template <class T>
void Launch<T>::prim(const Grid& g, double* U, T* W, unsigned long long* dtbits, unsigned* flags,
                     unsigned long long* floors, cudaStream_t s, T* Er) {
  k_prim<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, fields<8>(U, g.N), fields<8>(W, g.N), dtbits, flags, floors,
                                                fields<3>(Er, g.N));
}
template <class T>
void Launch<T>::flux_pcm(const Grid& g, int a, const T* W, const double* U, T* F, cudaStream_t s) {
  const dim3 gr = grid_of(g), bl(BX, BY);
  const Fields<const T, 8> Wf = fields<8>(W, g.N);
  const Fields<T, 7> Fa = fields<7>(F + a * 7 * g.N, g.N);
  const double* Ba = U + (5 + a) * g.N;
  if (a == 0) k_flux_pcm<T, 0><<<gr, bl, 0, s>>>(g, Wf, Ba, Fa);
  if (a == 1) k_flux_pcm<T, 1><<<gr, bl, 0, s>>>(g, Wf, Ba, Fa);
  if (a == 2) k_flux_pcm<T, 2><<<gr, bl, 0, s>>>(g, Wf, Ba, Fa);
}
template <class T, int RC>
static void launch_recon(const Grid& g, int a, const Fields<const T, 8>& W, const Fields<T, 7>& WL,
                         const Fields<T, 7>& WR, cudaStream_t s) {
  const dim3 gr = grid_of(g), bl(BX, BY);
  if (a == 0) k_recon<T, RC, 0><<<gr, bl, 0, s>>>(g, W, WL, WR);
  if (a == 1) k_recon<T, RC, 1><<<gr, bl, 0, s>>>(g, W, WL, WR);
  if (a == 2) k_recon<T, RC, 2><<<gr, bl, 0, s>>>(g, W, WL, WR);
}
template <class T>
void Launch<T>::recon(const Grid& g, int rc, int a, const T* W, T* WL, T* WR, cudaStream_t s) {
  const Fields<const T, 8> Wf = fields<8>(W, g.N);
  const Fields<T, 7> L = fields<7>(WL, g.N), R = fields<7>(WR, g.N);
  if (rc == 0) launch_recon<T, 0>(g, a, Wf, L, R, s);
  else if (rc == 1) launch_recon<T, 1>(g, a, Wf, L, R, s);
  else if (rc == 2) launch_recon<T, 2>(g, a, Wf, L, R, s);
  else launch_recon<T, 3>(g, a, Wf, L, R, s);
}
template <class T>
void Launch<T>::flux_hlld(const Grid& g, int a, const T* WL, const T* WR, const T* Bf, T* F, cudaStream_t s) {
  const dim3 gr = grid_of(g), bl(BX, BY);
  if constexpr (std::is_same<T, float>::value) {
    if (a == 0) k_flux_hlld_r<T, 0><<<gr, bl, 0, s>>>(g, WL, WR, Bf, F);
    if (a == 1) k_flux_hlld_r<T, 1><<<gr, bl, 0, s>>>(g, WL, WR, Bf, F);
    if (a == 2) k_flux_hlld_r<T, 2><<<gr, bl, 0, s>>>(g, WL, WR, Bf, F);
    return;
  }
  const Fields<const T, 7> L = fields<7>(WL, g.N), R = fields<7>(WR, g.N);
  const Fields<T, 7> Fa = fields<7>(F + a * 7 * g.N, g.N);
  const T* Ba = Bf + a * g.N;
  if (a == 0) k_flux_hlld<T, 0><<<gr, bl, 0, s>>>(g, L, R, Ba, Fa);
  if (a == 1) k_flux_hlld<T, 1><<<gr, bl, 0, s>>>(g, L, R, Ba, Fa);
  if (a == 2) k_flux_hlld<T, 2><<<gr, bl, 0, s>>>(g, L, R, Ba, Fa);
}
template <class T>
void Launch<T>::emf(const Grid& g, const T* W, const T* F, T* E, cudaStream_t s, const T* Er) {
  if constexpr (std::is_same<T, double>::value) {
    if (Er) k_emf_r<T, true><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, W, F, Er, E);
    else k_emf_r<T, false><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, W, F, Er, E);
    return;
  }
  const Fields<const T, 8> Wf = fields<8>(W, g.N);
  const Fields<const T, 21> Ff = fields<21>(F, g.N);
  const Fields<const T, 3> Rf = fields<3>(Er, g.N);
  const Fields<T, 3> Ef = fields<3>(E, g.N);
  if (Er) k_emf<T, true><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, Wf, Ff, Rf, Ef);
  else k_emf<T, false><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, Wf, Ff, Rf, Ef);
}
template <class T>
void Launch<T>::update_half(const Grid& g, const double* U, const T* F, const T* E, const double* dtp, T* W, T* Bh,
                            unsigned* flags, cudaStream_t s, T* Er) {
  k_update_half<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, fields<8>(U, g.N), fields<21>(F, g.N), fields<3>(E, g.N),
                                                       dtp, fields<8>(W, g.N), fields<3>(Bh, g.N), flags,
                                                       fields<3>(Er, g.N));
}
template <class T>
void Launch<T>::update_full(const Grid& g, double* U, const T* F, const T* E, const double* dtp, cudaStream_t s) {
  k_update_full<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, fields<8>(U, g.N), fields<21>(F, g.N), fields<3>(E, g.N),
                                                       dtp);
}
template <class T>
void Launch<T>::widen(const T* src, double* dst, long long n, cudaStream_t s) {
    k_widen<T><<<1216, 256, 0, s>>>(src, dst, n);
  }
template <class T>
void Launch<T>::narrow(const double* src, T* dst, long long n, cudaStream_t s) {
    k_narrow<T><<<1216, 256, 0, s>>>(src, dst, n);
  }

}  // namespace mhd
