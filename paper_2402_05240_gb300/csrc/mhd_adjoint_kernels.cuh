// mhd_adjoint_kernels.cuh -- the reverse sweep of one VL+CT step (not in the
// paper): gU^n = (dU^{n+1}/dU^n)^T gU^{n+1} at fixed dt, and the terms that
// make it the derivative of the step at the CFL dt of U^n (the dt cotangent
// from the two update reverses, the derivative of Eq. dt at its maximising
// cell).
//
// The forward intermediates are recomputed first (primitives W^n, predictor
// fluxes F^n, half-step state, interface states and corrector fluxes F^{n+1/2},
// edge fields).  The reverse kernels then run Step 9 back to Step 1.  Every
// reverse kernel is written in gather form: one thread owns one cell and only
// writes that cell's cotangents, reading the cotangents of its neighbours, so
// the result is deterministic (no floating-point atomics).  Cotangents of the
// state accumulate in double.
#pragma once

#include "mhd_adjoint.cuh"
#include "mhd_kernels.cuh"

namespace mhd {

template <class T> struct AdjBufs {
  // forward intermediates
  T *Wn, *Fn, *Wh, *Bh, *WLa, *WRa, *Fh, *Eh;
  double* Uh;  // [5][N] hydro half state
  // cotangents
  T *gF, *gE, *gW, *gWL, *gWR, *gS, *gBf, *gBcc, *gBccF;
  double* g5;  // [5][N]
};

// The reverse kernels address cells like the step kernels: 32-bit cell
// indices with the periodic neighbour offsets of thread_cell, and field
// pointers (fields()) formed once per thread from the restrict-qualified
// base pointers.
// the step scalars of a step of size dt (as the dt kernels form them)
__device__ __forceinline__ StepScalars step_scalars_of(const Grid& g, double dt) {
  StepScalars S;
  set_step_scalars(g, &S, dt);
  return S;
}

// ------------------------------------------------- R1: floors of Step 9 --
// Recomputes the pre-floor U^{n+1} of the cell; writes the pre-floor
// cotangent of the hydro fields into gU and the floor's B_cc cotangent.
template <class T>
__global__ void __launch_bounds__(BX* BY) k_adj_floors(Grid g, const double* __restrict__ U, const T* __restrict__ F,
                                                       const T* __restrict__ E, double dt,
                                                       const double* __restrict__ gUp, double* __restrict__ gU,
                                                       T* __restrict__ gBccF) {
  const Cell p = thread_cell(g);
  if (!p.ok) return;
  const long long N = g.N;
  const int c = p.c;
  const Fields<const double, 8> Uf = fields<8>(U, N);
  const Fields<const T, 21> Ff = fields<21>(F, N);
  const Fields<const T, 3> Ef = fields<3>(E, N);
  const StepScalars S = step_scalars_of(g, dt);
  double u5[5];
  constexpr bool X = Exact<T>::full;  // the arithmetic of k_update_full
  hydro_update<T, X, true, false>(Uf, Ff, S, p, u5);
  const double bx = face_update<T, X, true, 0>(g, Uf, Ef, S.dt, c, p.m[1], p.m[2]);
  const double by = face_update<T, X, true, 1>(g, Uf, Ef, S.dt, c, p.m[2], p.m[0]);
  const double bz = face_update<T, X, true, 2>(g, Uf, Ef, S.dt, c, p.m[0], p.m[1]);
  const double bxm = face_update<T, X, true, 0>(g, Uf, Ef, S.dt, c + p.m[0], p.m[1], p.m[2]);
  const double bym = face_update<T, X, true, 1>(g, Uf, Ef, S.dt, c + p.m[1], p.m[2], p.m[0]);
  const double bzm = face_update<T, X, true, 2>(g, Uf, Ef, S.dt, c + p.m[2], p.m[0], p.m[1]);
  const double b[3] = {0.5 * (bxm + bx), 0.5 * (bym + by), 0.5 * (bzm + bz)};
  double g5[5];
#pragma unroll
  for (int f = 0; f < 5; ++f) g5[f] = gUp[f * N + c];
  double gb[3] = {0.0, 0.0, 0.0};
  const bool rfl = u5[0] < g.rho_floor;
  const double r = rfl ? g.rho_floor : u5[0];
  const double ir = __drcp_rn(r);
  // kinetic + magnetic energy and the pressure-floor test with the forward's
  // arithmetic (k_prim; its FP32-bulk form in p_recover_f32)
  double ke, me;
  bool pfl;
  if constexpr (std::is_same<T, float>::value) {
    ke = 0.5 * ((u5[1] * u5[1] + u5[2] * u5[2] + u5[3] * u5[3]) * ir);
    me = 0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    const double bs[3] = {bxm + bx, bym + by, bzm + bz};
    double t2, pe;
    p_recover_f32(ir, u5[1], u5[2], u5[3], u5[4], bs, t2, pe);
    pfl = lt_pos<double>(g.gm1 * pe, g.p_floor);
  } else {
    ke = 0.5 * (u5[1] * (u5[1] * ir) + u5[2] * (u5[2] * ir) + u5[3] * (u5[3] * ir));
    me = 0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    pfl = g.gm1 * (u5[4] - ke - me) < g.p_floor;
  }
  if (pfl) {  // E = p_floor/(gamma-1) + |m|^2/(2 r) + |B_cc|^2/2
    const double gE = g5[4];
    g5[4] = 0.0;
    g5[1] += gE * u5[1] * ir;
    g5[2] += gE * u5[2] * ir;
    g5[3] += gE * u5[3] * ir;
    if (!rfl) g5[0] += -gE * ke * ir;
    gb[0] = gE * b[0];
    gb[1] = gE * b[1];
    gb[2] = gE * b[2];
  }
  if (rfl) g5[0] = 0.0;
#pragma unroll
  for (int f = 0; f < 5; ++f) gU[f * N + c] = g5[f];
  gBccF[c] = from_d<T>(gb[0]);
  gBccF[N + c] = from_d<T>(gb[1]);
  gBccF[2 * N + c] = from_d<T>(gb[2]);
}

// ------------------------------------------ R2 / R7: conservative update --
// U' = U - h div F, B' = B - h curl E.  Input: cotangents of the hydro U'
// (g5, own and upper neighbours) and of the faces (gface(p) computed by
// face_cot).  Output: gF hydro components, gE, and the identity part of gU.
// cotangent of the new face B_a of cell p: gUp face + (1/2)(gBcc_a(p) + gBcc_a(p + e_a))
template <class T, int A>
__device__ __forceinline__ double face_cot(const Grid& g, const double* __restrict__ gUpF, const T* __restrict__ gBcc,
                                           const T* __restrict__ gBfx, int q, int oA) {
  // q: the cell; oA: the offset from q to q + e_A
  const long long N = g.N;
  double v = 0.5 * (to_d<T>(gBcc[A * N + q]) + to_d<T>(gBcc[A * N + q + oA]));
  if (gUpF) v += gUpF[A * N + q];
  if (gBfx) v += to_d<T>(gBfx[A * N + q]);
  return v;
}

// Fixed-order block sum (shuffle tree, then the warps in order): one partial
// per block, so a later fixed-order sum of the partials is deterministic.
__device__ __forceinline__ void block_sum_to(double v, double* part) {
  __shared__ double red[BX * BY / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int t = threadIdx.y * BX + threadIdx.x;
  if ((t & 31) == 0) red[t >> 5] = v;
  __syncthreads();
  if (t == 0) {
    double m = red[0];
    for (int w = 1; w < BX * BY / 32; ++w) m += red[w];
    part[blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z)] = m;
  }
}

// d(update increment)/d(h) paired with the cotangents of the updated cell:
// sum_f g_f D_f + sum_a g_face_a curl_a, with D_f = sum_a (F_a(p) - F_a(p - e_a))/d_a
// and curl_a the face curl of E (the update is U' = U - h D, B' = B - h curl).
template <class T>
__device__ __forceinline__ double update_rate_dot(const Grid& g, const T* __restrict__ F, const T* __restrict__ E,
                                                  const double* g5, const double* gf, const Cell& p) {
  const long long N = g.N;
  const int c = p.c;
  double s = 0.0;
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    double d = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T* Fa = F + ((long long)a * 7 + comp_of(f, a)) * N;
      d += g.id[a] * (to_d<T>(Fa[c]) - to_d<T>(Fa[c + p.m[a]]));
    }
    s += g5[f] * d;
  }
  const Fields<const T, 3> Ef = fields<3>(E, N);
  s += gf[0] * face_curl<T, true, 0>(g, Ef, c, p.m[1], p.m[2]);
  s += gf[1] * face_curl<T, true, 1>(g, Ef, c, p.m[2], p.m[0]);
  s += gf[2] * face_curl<T, true, 2>(g, Ef, c, p.m[0], p.m[1]);
  return s;
}

// one cell of k_adj_update; returns its update_rate_dot term when SENS
template <class T, int MODE, bool SENS>
__device__ __forceinline__ double adj_update_cell(const Grid& g, double h, const double* g5src,
                                                  const double* __restrict__ gUpF, const T* __restrict__ gBcc,
                                                  const T* __restrict__ gBfx, double* gU, T* __restrict__ gF,
                                                  T* __restrict__ gE, const T* __restrict__ Fs,
                                                  const T* __restrict__ Es, const Cell& p) {
  const long long N = g.N;
  const int c = p.c;
  const int cp[3] = {c + p.p[0], c + p.p[1], c + p.p[2]};
  // hydro: U'_f(p) has -h/d_a F_a(p) and +h/d_a F_a(p - e_a), so
  // gF_a[comp](p) = -(h/d_a)(g_f(p) - g_f(p + e_a))
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T s = from_d<T>(-h * g.id[a]);
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      // (the difference of the double cotangents in double, the product in T)
      const double gv = g5src[f * N + c] - g5src[f * N + cp[a]];
      gF[((long long)a * 7 + comp_of(f, a)) * N + c] = from_d<T>(gv) * s;
    }
  }
  // faces of this cell and of the upper neighbours needed by the edge cotangents
  const double gf0 = face_cot<T, 0>(g, gUpF, gBcc, gBfx, c, p.p[0]);
  const double gf1 = face_cot<T, 1>(g, gUpF, gBcc, gBfx, c, p.p[1]);
  const double gf2 = face_cot<T, 2>(g, gUpF, gBcc, gBfx, c, p.p[2]);
  // E_k(q) enters B_{k+1}(q) with -h/d_{k+2}, B_{k+1}(q + e_{k+2}) with +h/d_{k+2},
  // B_{k+2}(q) with +h/d_{k+1}, B_{k+2}(q + e_{k+1}) with -h/d_{k+1}
  // neighbours' face cotangents
  const double f0_y = face_cot<T, 0>(g, gUpF, gBcc, gBfx, cp[1], p.p[0]);
  const double f0_z = face_cot<T, 0>(g, gUpF, gBcc, gBfx, cp[2], p.p[0]);
  const double f1_x = face_cot<T, 1>(g, gUpF, gBcc, gBfx, cp[0], p.p[1]);
  const double f1_z = face_cot<T, 1>(g, gUpF, gBcc, gBfx, cp[2], p.p[1]);
  const double f2_x = face_cot<T, 2>(g, gUpF, gBcc, gBfx, cp[0], p.p[2]);
  const double f2_y = face_cot<T, 2>(g, gUpF, gBcc, gBfx, cp[1], p.p[2]);
  const T hx = from_d<T>(h * g.id[0]), hy = from_d<T>(h * g.id[1]), hz = from_d<T>(h * g.id[2]);
  // k = 0 (E_x): B_y (a=1) with e_z, B_z (a=2) with e_y
  gE[c] = hy * from_d<T>(gf2 - f2_y) - hz * from_d<T>(gf1 - f1_z);
  // k = 1 (E_y): B_z with e_x, B_x with e_z
  gE[N + c] = hz * from_d<T>(gf0 - f0_z) - hx * from_d<T>(gf2 - f2_x);
  // k = 2 (E_z): B_x with e_y, B_y with e_x
  gE[2 * N + c] = hx * from_d<T>(gf1 - f1_x) - hy * from_d<T>(gf0 - f0_y);
  if (MODE == 0) {
    gU[5 * N + c] = gf0;
    gU[6 * N + c] = gf1;
    gU[7 * N + c] = gf2;
  } else {
#pragma unroll
    for (int f = 0; f < 5; ++f) gU[f * N + c] += g5src[f * N + c];
    gU[5 * N + c] += gf0;
    gU[6 * N + c] += gf1;
    gU[7 * N + c] += gf2;
  }
  if (SENS) {
    double g5[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) g5[f] = g5src[f * N + c];
    const double gf[3] = {gf0, gf1, gf2};
    return update_rate_dot<T>(g, Fs, Es, g5, gf, p);
  }
  return 0.0;
}

// MODE 0 (Step 9): gface from gUp faces + floor gBcc; writes gU faces = gface.
// MODE 1 (Step 5): gface from gBf (HLLD B_n) + gBcc (W^{n+1/2}); gU faces += gface.
// SENS: also the block partials of sum_p update_rate_dot(Fs, Es) (the
// cotangent of the step size h, up to the sign) into part.
template <class T, int MODE, bool SENS>
__global__ void __launch_bounds__(BX* BY) k_adj_update(Grid g, double h, const double* g5src,
                                                       const double* __restrict__ gUpF, const T* __restrict__ gBcc,
                                                       const T* __restrict__ gBfx, double* gU,
                                                       T* __restrict__ gF, T* __restrict__ gE,
                                                       const T* __restrict__ Fs, const T* __restrict__ Es,
                                                       double* __restrict__ part) {
  const Cell p = thread_cell(g);
  double sens = 0.0;
  if (p.ok) sens = adj_update_cell<T, MODE, SENS>(g, h, g5src, gUpF, gBcc, gBfx, gU, gF, gE, Fs, Es, p);
  if (SENS) block_sum_to(sens, part);
}

// Blocks per SM requested from the register allocator for the float-pair
// reverse HLLD and PPMC kernels (3: at most 168 registers; the reverse HLLD
// then spills about 1 KB per thread).  Measured, adjoint step of the 256^3
// turbulent box: 207.5 ms against 220.7 ms without the bound and 238.3 ms
// at 4 blocks; the float kernels are fastest without it (33.7 ms against
// 36.6 ms at 3 and 35.9 ms at 4 blocks).  0: no bound (the allocation of a
// plain __launch_bounds__(128)).
template <class T> struct AdjMinBlocks { static constexpr int v = 0; };
template <> struct AdjMinBlocks<df> { static constexpr int v = 3; };

// ---------------------------------------------------- R3 / R8: edge EMF --
// Gather-form reverse of Eq. emf-edge: writes gF[a][5], gF[a][6] and the
// reference-field part of gW (v and B_cc components; rho, P zeroed).  The
// arithmetic is in the compute type (the cotangents are stored in it).
template <class T> __device__ __forceinline__ T upw_lo_t(T m) {
  return m > T(0) ? T(1) : (m < T(0) ? T(0) : T(0.5));
}

template <class T, int K>
__device__ __forceinline__ void emf_cot_edge(const Grid& g, const T* __restrict__ W, const T* __restrict__ F,
                                             const T* __restrict__ gE, const Cell& p, T* __restrict__ gF,
                                             T* gW8) {
  constexpr int B = (K + 1) % 3, C = (K + 2) % 3;
  const long long N = g.N;
  // cell p + db e_B + dc e_C (|db|, |dc| <= 1; the wraps along B and C are independent)
  auto at = [&](int db, int dc) {
    return p.c + (db < 0 ? p.m[B] : (db > 0 ? p.p[B] : 0)) + (dc < 0 ? p.m[C] : (dc > 0 ? p.p[C] : 0));
  };
  const int c00 = at(0, 0), cb = at(-1, 0), cc = at(0, -1), cbc = at(-1, -1);
  const int cpb = at(1, 0), cpc = at(0, 1), cmcpb = at(1, -1), cmbpc = at(-1, 1);
  const T* Fb = F + (long long)B * 7 * N;  // mass flux of b-faces: Fb[x]
  const T* Fc = F + (long long)C * 7 * N;
  const T* gEk = gE + (long long)K * N;
  const T g00 = gEk[c00], gmb = gEk[cb], gmc = gEk[cc], gmbc = gEk[cbc];
  // upwind weights of the mass fluxes mc(q), mc(q + e_b), mc(q - e_c), mc(q - e_c + e_b);
  // mb(q), mb(q + e_c), mb(q - e_b), mb(q - e_b + e_c)
  const T uc0 = upw_lo_t<T>(Fc[c00]), uc_pb = upw_lo_t<T>(Fc[cpb]), uc_mc = upw_lo_t<T>(Fc[cc]),
          uc_mcpb = upw_lo_t<T>(Fc[cmcpb]);
  const T ub0 = upw_lo_t<T>(Fb[c00]), ub_pc = upw_lo_t<T>(Fb[cpc]), ub_mb = upw_lo_t<T>(Fb[cb]),
          ub_mbpc = upw_lo_t<T>(Fb[cmbpc]);
  const T q4 = T(0.25);
  const T gbf = q4 * g00 * (T(1) + uc_pb + uc0) + q4 * gmc * (T(1) + (T(1) - uc_mcpb) + (T(1) - uc_mc));
  const T gcf = q4 * g00 * (T(1) + ub_pc + ub0) + q4 * gmb * (T(1) + (T(1) - ub_mbpc) + (T(1) - ub_mb));
  const T grf = -q4 * (g00 * (uc0 + ub0) + gmb * (uc0 + (T(1) - ub_mb)) + gmc * ((T(1) - uc_mc) + ub0) +
                       gmbc * ((T(1) - uc_mc) + (T(1) - ub_mb)));
  // bf = -F_B[5], cf = +F_C[6]
  gF[((long long)B * 7 + 5) * N + c00] = -gbf;
  gF[((long long)C * 7 + 6) * N + c00] = gcf;
  // ref_K = -(v_B B_C - v_C B_B)
  const T vB = W[(1 + B) * N + c00], vC = W[(1 + C) * N + c00];
  const T BB = W[(5 + B) * N + c00], BC = W[(5 + C) * N + c00];
  gW8[1 + B] += -grf * BC;
  gW8[5 + C] += -grf * vB;
  gW8[1 + C] += grf * BB;
  gW8[5 + B] += grf * vC;
}

template <class T>
__global__ void __launch_bounds__(BX* BY) k_adj_emf(Grid g, const T* __restrict__ W, const T* __restrict__ F,
                                                    const T* __restrict__ gE, T* __restrict__ gF, T* __restrict__ gW) {
  const Cell p = thread_cell(g);
  if (!p.ok) return;
  const long long N = g.N;
  const int c = p.c;
  T gw[8] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  emf_cot_edge<T, 0>(g, W, F, gE, p, gF, gw);
  emf_cot_edge<T, 1>(g, W, F, gE, p, gF, gw);
  emf_cot_edge<T, 2>(g, W, F, gE, p, gF, gw);
#pragma unroll
  for (int f = 0; f < 8; ++f) gW[f * N + c] = gw[f];
}

// -------------------------------------------------- R4a / R9: HLLD reverse --
// PCM (predictor): states from W of cells p and p + e_A, B_n from U's face.
// Corrector: states from W_L, W_R buffers, B_n from the half-step faces.
// Writes gWL(p) (left state of face p), gWR(p + e_A) (right state of the
// face, owned by cell p + e_A) and gBf_A(p).
template <class T, int A, bool PCM>
__global__ void __launch_bounds__(BX* BY, AdjMinBlocks<T>::v) k_adj_hlld(Grid g, const T* __restrict__ WL, const T* __restrict__ WR,
                                                     const T* __restrict__ Wn, const double* __restrict__ U,
                                                     const T* __restrict__ Bh, const T* __restrict__ gF,
                                                     T* __restrict__ gWL, T* __restrict__ gWR, T* __restrict__ gBf) {
  const CellIdx ci = cell_of_thread(g);
  if (!ci.ok) return;
  const long long N = g.N, c = cidx(g, ci.i, ci.j, ci.k), cn = nb<A>(g, ci.i, ci.j, ci.k, 1);
  T wl[7], wr[7], gf[7], gwl[7], gwr[7];
  T bn;
  if (PCM) {
    load_dir<A>(Wn, N, c, wl);
    load_dir<A>(Wn, N, cn, wr);
    bn = from_d<T>(U[(5 + A) * N + c]);
  } else {
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      wl[q] = WL[q * N + c];
      wr[q] = WR[q * N + cn];
    }
    bn = Bh[A * N + c];
  }
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    gf[q] = gF[((long long)A * 7 + q) * N + c];
    gwl[q] = gwr[q] = T(0);
  }
  T gbn = T(0);
  hlld_vjp<T>(from_d<T>(g.gamma), wl, wr, bn, gf, gwl, gwr, gbn);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    gWL[q * N + c] = gwl[q];
    gWR[q * N + cn] = gwr[q];
  }
  gBf[A * N + c] = gbn;
}

// directional 7-vector cotangent -> W field cotangents (accumulate)
template <int A, class T> __device__ __forceinline__ void add_dir(T* __restrict__ gW, long long N, long long q, const T* gw) {
  constexpr int B = (A + 1) % 3, C = (A + 2) % 3;
  gW[q] += gw[0];
  gW[(1 + A) * N + q] += gw[1];
  gW[(1 + B) * N + q] += gw[2];
  gW[(1 + C) * N + q] += gw[3];
  gW[4 * N + q] += gw[4];
  gW[(5 + B) * N + q] += gw[5];
  gW[(5 + C) * N + q] += gw[6];
}

// predictor: both face-state cotangents of cell p belong to cell p itself
template <class T, int A>
__global__ void __launch_bounds__(BX* BY) k_adj_pcm_gather(Grid g, const T* __restrict__ gWL, const T* __restrict__ gWR,
                                                           T* __restrict__ gW) {
  const CellIdx ci = cell_of_thread(g);
  if (!ci.ok) return;
  const long long N = g.N, c = cidx(g, ci.i, ci.j, ci.k);
  T s[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) s[q] = gWL[q * N + c] + gWR[q * N + c];
  add_dir<A>(gW, N, c, s);
}

// ------------------------------------------------- R4b/c: reconstruction --
// Per cell: reverse of PLMC / PPMC for axis A; slots S[m][7] for the stencil
// cells (PLMC m = 0..2 for p-1..p+1, PPMC m = 0..4 for p-2..p+2) and
// S[NS*7] for the cotangent of the cell-centred B_A of cell p.
template <class T, int RECON, int A>
__global__ void __launch_bounds__(BX* BY) k_adj_recon(Grid g, const T* __restrict__ W, const T* __restrict__ gWL,
                                                      const T* __restrict__ gWR, T* __restrict__ S) {
  const CellIdx ci = cell_of_thread(g);
  if (!ci.ok) return;
  const long long N = g.N, c = cidx(g, ci.i, ci.j, ci.k);
  constexpr int NS = RECON == 2 ? 5 : 3;
  T gl[7], gr[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    gl[q] = gWL[q * N + c];
    gr[q] = gWR[q * N + c];
  }
  const T bn = W[(5 + A) * N + c];
  T gbn = T(0);
  T gw[NS][7];
#pragma unroll
  for (int m = 0; m < NS; ++m)
#pragma unroll
    for (int q = 0; q < 7; ++q) gw[m][q] = T(0);
  if constexpr (RECON == 0) {
    // W_L = W_R = W_p, with the face floors
    T w0[7];
    load_dir<A>(W, N, c, w0);
#pragma unroll
    for (int q = 0; q < 7; ++q) {
      T a = gl[q], b = gr[q];
      if (q == 0 && w0[0] < from_d<T>(g.rho_floor)) a = b = T(0);
      if (q == 4 && w0[4] < from_d<T>(g.p_floor)) a = b = T(0);
      gw[1][q] = a + b;
    }
  } else if constexpr (RECON == 1) {
    T wm[7], w0[7], wp[7];
    load_dir<A>(W, N, nb<A>(g, ci.i, ci.j, ci.k, -1), wm);
    load_dir<A>(W, N, c, w0);
    load_dir<A>(W, N, nb<A>(g, ci.i, ci.j, ci.k, 1), wp);
    plmc_vjp<T>(from_d<T>(g.gamma), from_d<T>(g.rho_floor), from_d<T>(g.p_floor), wm, w0, wp, bn, gl, gr, gw[0], gw[1],
                gw[2], gbn);
  } else {
    // stencil cells loaded where the reverse sweep uses them (from L1), the
    // slots of the neighbours written as they are formed
    auto wload = [&](int m, T* out) { load_dir<A>(W, N, nb<A>(g, ci.i, ci.j, ci.k, m - 2), out); };
    auto put = [&](int m, const T* gm) {
#pragma unroll
      for (int q = 0; q < 7; ++q) S[((long long)m * 7 + q) * N + c] = gm[q];
    };
    T gw2[7];
    ppmc_vjp<T>(from_d<T>(g.gamma), from_d<T>(g.rho_floor), from_d<T>(g.p_floor), wload, bn, gl, gr, put, gw2, gbn);
    put(2, gw2);
    S[(long long)NS * 7 * N + c] = gbn;
    return;
  }
#pragma unroll
  for (int m = 0; m < NS; ++m)
#pragma unroll
    for (int q = 0; q < 7; ++q) S[((long long)m * 7 + q) * N + c] = gw[m][q];
  S[(long long)NS * 7 * N + c] = gbn;
}

// PPMC reverse in three passes (ppmc_vjp_pass1..3).  X (kPpmcRevFields
// arrays) carries gdm, gdp, the 17 eigensystem cotangents and the cell's own
// cotangent from pass 1 to passes 2 and 3; pass 2 writes its deviation
// cotangents into the slots of S that pass 3 then overwrites with the
// stencil cells' cotangents (each cell's slots are read and written by its
// own thread only).  S has the slot layout of k_adj_recon.
template <class T, int A>
__global__ void __launch_bounds__(BX* BY, AdjMinBlocks<T>::v) k_adj_ppmc1(Grid g, const T* __restrict__ W, const T* __restrict__ gWL,
                                                      const T* __restrict__ gWR, Fields<T, kPpmcRevFields> X) {
  const CellIdx ci = cell_of_thread(g);
  if (!ci.ok) return;
  const long long N = g.N, c = cidx(g, ci.i, ci.j, ci.k);
  T gl[7], gr[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    gl[q] = gWL[q * N + c];
    gr[q] = gWR[q * N + c];
  }
  const T bn = W[(5 + A) * N + c];
  auto wload = [&](int m, T* out) { load_dir<A>(W, N, nb<A>(g, ci.i, ci.j, ci.k, m - 2), out); };
  T gdm[7], gdp[7], gw2[7], ge[17];
  EigG<T> gE;
  ppmc_vjp_pass1<T>(from_d<T>(g.gamma), from_d<T>(g.rho_floor), from_d<T>(g.p_floor), wload, bn, gl, gr, gdm, gdp,
                    gE, gw2);
  eigg_pack<T>(gE, ge);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    X.f[q][c] = gdm[q];
    X.f[7 + q][c] = gdp[q];
    X.f[31 + q][c] = gw2[q];
  }
#pragma unroll
  for (int q = 0; q < 17; ++q) X.f[14 + q][c] = ge[q];
}

template <class T, int A>
__global__ void __launch_bounds__(BX* BY, AdjMinBlocks<T>::v) k_adj_ppmc2(Grid g, const T* __restrict__ W, Fields<T, kPpmcRevFields> X,
                                                      T* __restrict__ S) {
  const CellIdx ci = cell_of_thread(g);
  if (!ci.ok) return;
  const long long N = g.N, c = cidx(g, ci.i, ci.j, ci.k);
  T gdm[7], gdp[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    gdm[q] = X.f[q][c];
    gdp[q] = X.f[7 + q][c];
  }
  const T bn = W[(5 + A) * N + c];
  auto wload = [&](int m, T* out) { load_dir<A>(W, N, nb<A>(g, ci.i, ci.j, ci.k, m - 2), out); };
  T gq[4][7];
  ppmc_vjp_pass2<T>(from_d<T>(g.gamma), wload, bn, gdm, gdp, gq);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int m = k < 2 ? k : k + 1;
#pragma unroll
    for (int q = 0; q < 7; ++q) S[((long long)m * 7 + q) * N + c] = gq[k][q];
  }
}

template <class T, int A>
__global__ void __launch_bounds__(BX* BY, AdjMinBlocks<T>::v) k_adj_ppmc3(Grid g, const T* __restrict__ W, Fields<T, kPpmcRevFields> X,
                                                      T* __restrict__ S) {
  const CellIdx ci = cell_of_thread(g);
  if (!ci.ok) return;
  const long long N = g.N, c = cidx(g, ci.i, ci.j, ci.k);
  T gw2[7], ge[17];
#pragma unroll
  for (int q = 0; q < 7; ++q) gw2[q] = X.f[31 + q][c];
#pragma unroll
  for (int q = 0; q < 17; ++q) ge[q] = X.f[14 + q][c];
  EigG<T> gE;
  eigg_unpack<T>(ge, gE);
  const T bn = W[(5 + A) * N + c];
  auto wload = [&](int m, T* out) { load_dir<A>(W, N, nb<A>(g, ci.i, ci.j, ci.k, m - 2), out); };
  auto gqload = [&](int k, T* out) {
    const int m = k < 2 ? k : k + 1;
#pragma unroll
    for (int q = 0; q < 7; ++q) out[q] = S[((long long)m * 7 + q) * N + c];
  };
  auto put = [&](int m, const T* gm) {
#pragma unroll
    for (int q = 0; q < 7; ++q) S[((long long)m * 7 + q) * N + c] = gm[q];
  };
  T gbn = T(0);
  ppmc_vjp_pass3<T>(from_d<T>(g.gamma), wload, bn, gqload, gE, gw2, put, gbn);
#pragma unroll
  for (int q = 0; q < 7; ++q) S[(2LL * 7 + q) * N + c] = gw2[q];
  S[5LL * 7 * N + c] = gbn;
}

// Passes 2 and 3 in one kernel, the deviation cotangents kept in registers
// (for the float reverse, whose live state fits without spilling).
template <class T, int A>
__global__ void __launch_bounds__(BX* BY, AdjMinBlocks<T>::v) k_adj_ppmc23(Grid g, const T* __restrict__ W,
                                                                          Fields<T, kPpmcRevFields> X,
                                                                          T* __restrict__ S) {
  const CellIdx ci = cell_of_thread(g);
  if (!ci.ok) return;
  const long long N = g.N, c = cidx(g, ci.i, ci.j, ci.k);
  T gdm[7], gdp[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    gdm[q] = X.f[q][c];
    gdp[q] = X.f[7 + q][c];
  }
  const T bn = W[(5 + A) * N + c];
  auto wload = [&](int m, T* out) { load_dir<A>(W, N, nb<A>(g, ci.i, ci.j, ci.k, m - 2), out); };
  T gq[4][7];
  ppmc_vjp_pass2<T>(from_d<T>(g.gamma), wload, bn, gdm, gdp, gq);
  T gw2[7], ge[17];
#pragma unroll
  for (int q = 0; q < 7; ++q) gw2[q] = X.f[31 + q][c];
#pragma unroll
  for (int q = 0; q < 17; ++q) ge[q] = X.f[14 + q][c];
  EigG<T> gE;
  eigg_unpack<T>(ge, gE);
  auto gqload = [&](int k, T* out) {
#pragma unroll
    for (int q = 0; q < 7; ++q) out[q] = gq[k][q];
  };
  auto put = [&](int m, const T* gm) {
#pragma unroll
    for (int q = 0; q < 7; ++q) S[((long long)m * 7 + q) * N + c] = gm[q];
  };
  T gbn = T(0);
  ppmc_vjp_pass3<T>(from_d<T>(g.gamma), wload, bn, gqload, gE, gw2, put, gbn);
#pragma unroll
  for (int q = 0; q < 7; ++q) S[(2LL * 7 + q) * N + c] = gw2[q];
  S[5LL * 7 * N + c] = gbn;
}

// cell p gathers slot m from cell p - (m - h) along A, h = NS/2
template <class T, int RECON, int A>
__global__ void __launch_bounds__(BX* BY) k_adj_recon_gather(Grid g, const T* __restrict__ S, T* __restrict__ gW) {
  const CellIdx ci = cell_of_thread(g);
  if (!ci.ok) return;
  const long long N = g.N, c = cidx(g, ci.i, ci.j, ci.k);
  constexpr int NS = RECON == 2 ? 5 : 3;
  constexpr int H = NS / 2;
  T acc[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int m = 0; m < NS; ++m) {
    // the owner o has this cell at offset (m - H): o = p - (m - H)
    const long long o = nb<A>(g, ci.i, ci.j, ci.k, H - m);
#pragma unroll
    for (int q = 0; q < 7; ++q) acc[q] += S[((long long)m * 7 + q) * N + o];
  }
  add_dir<A>(gW, N, c, acc);
  gW[(5 + A) * N + c] += S[(long long)NS * 7 * N + c];
}

// ------------------------------------------------ R5 / R10: primitives --
// W = prim(hydro, B_cc): cotangent of the hydro fields (g5 out) and of B_cc
// (gBcc out).  HALF: hydro from the stored half state; else from U^n.
template <class T, bool HALF>
__global__ void __launch_bounds__(BX* BY) k_adj_prim(Grid g, const double* __restrict__ U, const double* __restrict__ Uh,
                                                     const T* __restrict__ Bh, const T* __restrict__ gW,
                                                     double* __restrict__ g5, T* __restrict__ gBcc) {
  const Cell p = thread_cell(g);
  if (!p.ok) return;
  const long long N = g.N;
  const int c = p.c;
  double h5[5], b[3];
  if (HALF) {
#pragma unroll
    for (int f = 0; f < 5; ++f) h5[f] = Uh[f * N + c];
    b[0] = 0.5 * (to_d<T>(Bh[c + p.m[0]]) + to_d<T>(Bh[c]));
    b[1] = 0.5 * (to_d<T>(Bh[N + c + p.m[1]]) + to_d<T>(Bh[N + c]));
    b[2] = 0.5 * (to_d<T>(Bh[2 * N + c + p.m[2]]) + to_d<T>(Bh[2 * N + c]));
  } else {
#pragma unroll
    for (int f = 0; f < 5; ++f) h5[f] = U[f * N + c];
    b[0] = 0.5 * (U[5 * N + c + p.m[0]] + U[5 * N + c]);
    b[1] = 0.5 * (U[6 * N + c + p.m[1]] + U[6 * N + c]);
    b[2] = 0.5 * (U[7 * N + c + p.m[2]] + U[7 * N + c]);
  }
  if constexpr (std::is_same<T, float>::value) {
    float gw8[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) gw8[f] = gW[f * N + c];
    float o5[5], gb[3];
    prim_vjp_f32(g, h5[0], h5[1], h5[2], h5[3], h5[4], b, gw8, o5, gb);
#pragma unroll
    for (int f = 0; f < 5; ++f) g5[f * N + c] = f2d_bits(o5[f]);
    gBcc[c] = gb[0];
    gBcc[N + c] = gb[1];
    gBcc[2 * N + c] = gb[2];
  } else {
    double gw8[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) gw8[f] = to_d<T>(gW[f * N + c]);
    double o5[5], gb[3] = {0.0, 0.0, 0.0};
    prim_vjp(g, h5[0], h5[1], h5[2], h5[3], h5[4], b, gw8, o5, gb);
#pragma unroll
    for (int f = 0; f < 5; ++f) g5[f * N + c] = o5[f];
    gBcc[c] = from_d<T>(gb[0]);
    gBcc[N + c] = from_d<T>(gb[1]);
    gBcc[2 * N + c] = from_d<T>(gb[2]);
  }
}

// R11: predictor faces: gU faces += gBf_a(p) + (1/2)(gBcc_a(p) + gBcc_a(p + e_a)); gU hydro += g5
template <class T>
__global__ void __launch_bounds__(BX* BY) k_adj_faces_n(Grid g, const double* __restrict__ g5, const T* __restrict__ gBcc,
                                                        const T* __restrict__ gBf, double* __restrict__ gU) {
  const Cell p = thread_cell(g);
  if (!p.ok) return;
  const long long N = g.N;
  const int c = p.c;
#pragma unroll
  for (int f = 0; f < 5; ++f) gU[f * N + c] += g5[f * N + c];
  gU[5 * N + c] += face_cot<T, 0>(g, nullptr, gBcc, gBf, c, p.p[0]);
  gU[6 * N + c] += face_cot<T, 1>(g, nullptr, gBcc, gBf, c, p.p[1]);
  gU[7 * N + c] += face_cot<T, 2>(g, nullptr, gBcc, gBf, c, p.p[2]);
}

// forward half update that also keeps the hydro half state (for R5)
template <class T>
__global__ void __launch_bounds__(BX* BY) k_fwd_half_keep(Grid g, const double* __restrict__ U0, const T* __restrict__ F,
                                                          const T* __restrict__ E, double dt, T* __restrict__ W,
                                                          T* __restrict__ Bh, double* __restrict__ Uh) {
  const Cell p = thread_cell(g);
  if (!p.ok) return;
  const long long N = g.N;
  const int c = p.c;
  const Fields<const double, 8> Uf = fields<8>(U0, N);
  const Fields<const T, 21> Ff = fields<21>(F, N);
  const Fields<const T, 3> Ef = fields<3>(E, N);
  const StepScalars S = step_scalars_of(g, dt);
  const double h = S.h_half;
  constexpr bool X = sizeof(T) == 8 && Exact<T>::full;  // the arithmetic of k_update_half
  double u5[5];
  hydro_update<T, X, true, true>(Uf, Ff, S, p, u5);
  const double bx = face_update<T, X, true, 0>(g, Uf, Ef, h, c, p.m[1], p.m[2]);
  const double by = face_update<T, X, true, 1>(g, Uf, Ef, h, c, p.m[2], p.m[0]);
  const double bz = face_update<T, X, true, 2>(g, Uf, Ef, h, c, p.m[0], p.m[1]);
  const double bxm = face_update<T, X, true, 0>(g, Uf, Ef, h, c + p.m[0], p.m[1], p.m[2]);
  const double bym = face_update<T, X, true, 1>(g, Uf, Ef, h, c + p.m[1], p.m[2], p.m[0]);
  const double bzm = face_update<T, X, true, 2>(g, Uf, Ef, h, c + p.m[2], p.m[0], p.m[1]);
  Bh[c] = from_d<T>(bx);
  Bh[N + c] = from_d<T>(by);
  Bh[2 * N + c] = from_d<T>(bz);
#pragma unroll
  for (int f = 0; f < 5; ++f) Uh[f * N + c] = u5[f];
  const double bcc[3] = {0.5 * (bxm + bx), 0.5 * (bym + by), 0.5 * (bzm + bz)};
  const PrimD pw = prim_core(g, u5[0], u5[1], u5[2], u5[3], u5[4], bcc);
  T w8[8];
  store_w<T>(fields<8>(W, N), c, pw, w8);
}

// ------------------------------------- the CFL dt as a function of U^n --
// dt(U) = C_CFL / r_max, r_max = max over cells p and axes l of
// (|v_l| + c_f,l)(p) / d_l (Eq. dt, Step 1).  Its reverse adds
// g_dt * d dt/dU to gU, where g_dt = <gU^{n+1}, dU^{n+1}/d dt> =
// -sum_p [update_rate_dot of Step 9 + 1/2 update_rate_dot of Step 5], and
// d dt/dU = -(dt / r_max) d r_max/dU is nonzero only at the maximising cell.
// The maximum is differentiated at the lowest cell index reaching it (then
// the lowest axis): one element of the subdifferential where cells tie.

// c_f of Eq. c_f on forward-mode numbers (the formula of fast_speed)
__device__ __forceinline__ Dl<double> fast_speed_dl(double gamma, Dl<double> rho, Dl<double> p, Dl<double> bl,
                                                    Dl<double> bt1, Dl<double> bt2) {
  const Dl<double> ir = Dl<double>(1.0) / rho;
  const Dl<double> a2 = Dl<double>(gamma) * p * ir;
  const Dl<double> t2 = (bt1 * bt1 + bt2 * bt2) * ir;
  const Dl<double> b2 = bl * bl * ir + t2;
  const Dl<double> dd = a2 - b2;
  return dsqrt(Dl<double>(0.5) * (a2 + b2 + dsqrt(dd * dd + Dl<double>(4.0) * a2 * t2)));
}

// cells whose inverse crossing time (computed as in k_prim) equals r_max
// post their index; the integer minimum is the maximising cell
template <class T>
__global__ void __launch_bounds__(BX* BY) k_adj_cfl_argmax(Grid g, const T* __restrict__ W,
                                                           const unsigned long long* __restrict__ rbits,
                                                           unsigned long long* __restrict__ idx) {
  const CellIdx ci = cell_of_thread(g);
  if (!ci.ok || !interior(g, ci.i, ci.j, ci.k)) return;
  const long long N = g.N, c = cidx(g, ci.i, ci.j, ci.k);
  T w8[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) w8[f] = W[f * N + c];
  const double r = to_d<T>(cell_inv_crossing<T>(g, w8));
  if ((unsigned long long)__double_as_longlong(r) == *rbits) atomicMin(idx, (unsigned long long)c);
}

// one block: g_dt from the partials of both update reverses (fixed order),
// then d dt/dU at the maximising cell into gU.  out = {g_dt, dt, cell}.
constexpr int kCflThreads = 256;
template <class T>  // (instantiated once per compute type's translation unit)
__global__ void __launch_bounds__(kCflThreads) k_adj_cfl_term(Grid g, const double* __restrict__ U,
                                                              const double* __restrict__ part, long long nparts,
                                                              const unsigned long long* __restrict__ rbits,
                                                              const unsigned long long* __restrict__ idx,
                                                              double* __restrict__ gU, double* __restrict__ out) {
  __shared__ double red[kCflThreads];
  const int t = threadIdx.x;
  double acc = 0.0;
  for (long long q = t; q < nparts; q += kCflThreads) acc += part[q] + 0.5 * part[nparts + q];
  red[t] = acc;
  __syncthreads();
  for (int w = kCflThreads / 2; w > 0; w >>= 1) {
    if (t < w) red[t] += red[t + w];
    __syncthreads();
  }
  if (t != 0) return;
  const double gdt = -red[0];
  const double rmax = __longlong_as_double((long long)*rbits);
  const double dt = g.cfl / rmax;
  out[0] = gdt;
  out[1] = dt;
  out[2] = -1.0;
  const unsigned long long cu = *idx;
  if (cu >= (unsigned long long)g.N || !(rmax > 0.0)) return;
  const long long N = g.N, c = (long long)cu;
  const int i = (int)(c % g.n[0]), j = (int)((c / g.n[0]) % g.n[1]), k = (int)(c / ((long long)g.n[0] * g.n[1]));
  const long long cm[3] = {nb<0>(g, i, j, k, -1), nb<1>(g, i, j, k, -1), nb<2>(g, i, j, k, -1)};
  double b[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) b[a] = 0.5 * (U[(5 + a) * N + cm[a]] + U[(5 + a) * N + c]);
  const double r0 = U[c], m[3] = {U[N + c], U[2 * N + c], U[3 * N + c]}, e = U[4 * N + c];
  const PrimD p = prim_core(g, r0, m[0], m[1], m[2], e, b);
  // the axis of the maximum (first on ties), in double
  int l = 0;
  double best = -1.0;
  for (int a = 0; a < 3; ++a) {
    const double cf = fast_speed_dl(g.gamma, Dl<double>(p.rho), Dl<double>(p.p), Dl<double>(p.b[a]),
                                    Dl<double>(p.b[(a + 1) % 3]), Dl<double>(p.b[(a + 2) % 3])).v;
    const double ra = (fabs(p.v[a]) + cf) * g.id[a];
    if (ra > best) {
      best = ra;
      l = a;
    }
  }
  // d r / d (rho, P, B_l, B_t1, B_t2): one forward-mode pass per input
  double dcf[5];
  for (int q = 0; q < 5; ++q) {
    const Dl<double> x0(p.rho, q == 0 ? 1.0 : 0.0), x1(p.p, q == 1 ? 1.0 : 0.0), x2(p.b[l], q == 2 ? 1.0 : 0.0),
        x3(p.b[(l + 1) % 3], q == 3 ? 1.0 : 0.0), x4(p.b[(l + 2) % 3], q == 4 ? 1.0 : 0.0);
    dcf[q] = fast_speed_dl(g.gamma, x0, x1, x2, x3, x4).d;
  }
  const double coef = gdt * (-dt / rmax) * g.id[l];
  double gw8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  gw8[0] = coef * dcf[0];
  gw8[1 + l] = coef * (p.v[l] > 0.0 ? 1.0 : (p.v[l] < 0.0 ? -1.0 : 0.0));
  gw8[4] = coef * dcf[1];
  gw8[5 + l] = coef * dcf[2];
  gw8[5 + (l + 1) % 3] = coef * dcf[3];
  gw8[5 + (l + 2) % 3] = coef * dcf[4];
  double o5[5], gb[3] = {0.0, 0.0, 0.0};
  prim_vjp(g, r0, m[0], m[1], m[2], e, b, gw8, o5, gb);
#pragma unroll
  for (int f = 0; f < 5; ++f) gU[f * N + c] += o5[f];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gU[(5 + a) * N + c] += 0.5 * gb[a];
    gU[(5 + a) * N + cm[a]] += 0.5 * gb[a];
  }
  out[2] = (double)c;
}

// ---------------------------------------------- batch HLLD VJP (testing) --
template <class T>
__global__ void k_hlld_vjp_batch(int n, double gamma, const double* __restrict__ wl, const double* __restrict__ wr,
                                 const double* __restrict__ bn, const double* __restrict__ gf, double* __restrict__ gwl,
                                 double* __restrict__ gwr, double* __restrict__ gbn, double* __restrict__ f) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  T a[7], b[7], g[7], ga[7], gb[7], ff[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    a[q] = T(wl[7 * t + q]);
    b[q] = T(wr[7 * t + q]);
    g[q] = T(gf[7 * t + q]);
    ga[q] = gb[q] = T(0);
  }
  T gn = T(0);
  hlld_vjp<T>(T(gamma), a, b, T(bn[t]), g, ga, gb, gn);
  hlld<T>(T(gamma), T(1.0 / (gamma - 1.0)), a, b, T(bn[t]), ff);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    gwl[7 * t + q] = to_d<T>(ga[q]);
    gwr[7 * t + q] = to_d<T>(gb[q]);
    f[7 * t + q] = to_d<T>(ff[q]);
  }
  gbn[t] = to_d<T>(gn);
}

// --------------------------------------------------------------- launchers --

template <class T>
void AdjLaunch<T>::floors(const Grid& g, const double* U, const T* F, const T* E, double dt, const double* gUp, double* gU,
                     T* gBccF, cudaStream_t s) {
    k_adj_floors<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, U, F, E, dt, gUp, gU, gBccF);
  }
template <class T>
void AdjLaunch<T>::update(const Grid& g, int mode, double h, const double* g5src, const double* gUpF, const T* gBcc,
                     const T* gBfx, double* gU, T* gF, T* gE, cudaStream_t s, const T* Fs, const T* Es,
                     double* part) {
    const dim3 gr = grid_of(g), bl(BX, BY);
    if (part) {
      if (mode == 0)
        k_adj_update<T, 0, true><<<gr, bl, 0, s>>>(g, h, g5src, gUpF, gBcc, gBfx, gU, gF, gE, Fs, Es, part);
      else
        k_adj_update<T, 1, true><<<gr, bl, 0, s>>>(g, h, g5src, gUpF, gBcc, gBfx, gU, gF, gE, Fs, Es, part);
    } else {
      if (mode == 0)
        k_adj_update<T, 0, false><<<gr, bl, 0, s>>>(g, h, g5src, gUpF, gBcc, gBfx, gU, gF, gE, nullptr, nullptr,
                                                     nullptr);
      else
        k_adj_update<T, 1, false><<<gr, bl, 0, s>>>(g, h, g5src, gUpF, gBcc, gBfx, gU, gF, gE, nullptr, nullptr,
                                                     nullptr);
    }
  }
template <class T>
void AdjLaunch<T>::cfl_term(const Grid& g, const double* U, const T* W, const unsigned long long* rbits,
                            const double* part, long long nparts, unsigned long long* idx, double* gU, double* out,
                            cudaStream_t s) {
    cudaMemsetAsync(idx, 0xff, sizeof(unsigned long long), s);
    k_adj_cfl_argmax<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, W, rbits, idx);
    k_adj_cfl_term<T><<<1, kCflThreads, 0, s>>>(g, U, part, nparts, rbits, idx, gU, out);
  }
template <class T>
void AdjLaunch<T>::emf(const Grid& g, const T* W, const T* F, const T* gE, T* gF, T* gW, cudaStream_t s) {
    k_adj_emf<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, W, F, gE, gF, gW);
  }
template <class T>
void AdjLaunch<T>::hlld(const Grid& g, int a, bool pcm, const T* WL, const T* WR, const T* Wn, const double* U, const T* Bh,
                   const T* gF, T* gWL, T* gWR, T* gBf, cudaStream_t s) {
    const dim3 gr = grid_of(g), bl(BX, BY);
    if (pcm) {
      if (a == 0) k_adj_hlld<T, 0, true><<<gr, bl, 0, s>>>(g, WL, WR, Wn, U, Bh, gF, gWL, gWR, gBf);
      if (a == 1) k_adj_hlld<T, 1, true><<<gr, bl, 0, s>>>(g, WL, WR, Wn, U, Bh, gF, gWL, gWR, gBf);
      if (a == 2) k_adj_hlld<T, 2, true><<<gr, bl, 0, s>>>(g, WL, WR, Wn, U, Bh, gF, gWL, gWR, gBf);
    } else {
      if (a == 0) k_adj_hlld<T, 0, false><<<gr, bl, 0, s>>>(g, WL, WR, Wn, U, Bh, gF, gWL, gWR, gBf);
      if (a == 1) k_adj_hlld<T, 1, false><<<gr, bl, 0, s>>>(g, WL, WR, Wn, U, Bh, gF, gWL, gWR, gBf);
      if (a == 2) k_adj_hlld<T, 2, false><<<gr, bl, 0, s>>>(g, WL, WR, Wn, U, Bh, gF, gWL, gWR, gBf);
    }
  }
template <class T>
void AdjLaunch<T>::pcm_gather(const Grid& g, int a, const T* gWL, const T* gWR, T* gW, cudaStream_t s) {
    const dim3 gr = grid_of(g), bl(BX, BY);
    if (a == 0) k_adj_pcm_gather<T, 0><<<gr, bl, 0, s>>>(g, gWL, gWR, gW);
    if (a == 1) k_adj_pcm_gather<T, 1><<<gr, bl, 0, s>>>(g, gWL, gWR, gW);
    if (a == 2) k_adj_pcm_gather<T, 2><<<gr, bl, 0, s>>>(g, gWL, gWR, gW);
  }
// Which compute types take the three-pass PPMC reverse (else one kernel).
// Measured, adjoint step of the 256^3 turbulent box: float pairs 317 ->
// 222 ms (one kernel: 230 registers and a 1 KB stack frame, 2 blocks per
// SM), float 36.6 -> 34.2 ms; double 505 ms in one kernel against 536 ms in
// three (it recomputes the eigensystem and the deviations on the FP64 pipe).
template <class T> struct SplitPpmcRev { static constexpr bool v = !std::is_same<T, double>::value; };

template <class T, int A>
static void launch_ppmc_rev(const Grid& g, const T* W, const T* gWL, const T* gWR, T* S, T* gW,
                            const Fields<T, kPpmcRevFields>& X, cudaStream_t s) {
  const dim3 gr = grid_of(g), bl(BX, BY);
  k_adj_ppmc1<T, A><<<gr, bl, 0, s>>>(g, W, gWL, gWR, X);
  if constexpr (std::is_same<T, float>::value) {
    k_adj_ppmc23<T, A><<<gr, bl, 0, s>>>(g, W, X, S);
  } else {
    k_adj_ppmc2<T, A><<<gr, bl, 0, s>>>(g, W, X, S);
    k_adj_ppmc3<T, A><<<gr, bl, 0, s>>>(g, W, X, S);
  }
  k_adj_recon_gather<T, 2, A><<<gr, bl, 0, s>>>(g, S, gW);
}
template <class T>
template <int R>
void AdjLaunch<T>::recon_r(const Grid& g, int a, const T* W, const T* gWL, const T* gWR, T* S, T* gW,
                                       cudaStream_t s) {
    const dim3 gr = grid_of(g), bl(BX, BY);
    if (a == 0) {
      k_adj_recon<T, R, 0><<<gr, bl, 0, s>>>(g, W, gWL, gWR, S);
      k_adj_recon_gather<T, R, 0><<<gr, bl, 0, s>>>(g, S, gW);
    }
    if (a == 1) {
      k_adj_recon<T, R, 1><<<gr, bl, 0, s>>>(g, W, gWL, gWR, S);
      k_adj_recon_gather<T, R, 1><<<gr, bl, 0, s>>>(g, S, gW);
    }
    if (a == 2) {
      k_adj_recon<T, R, 2><<<gr, bl, 0, s>>>(g, W, gWL, gWR, S);
      k_adj_recon_gather<T, R, 2><<<gr, bl, 0, s>>>(g, S, gW);
    }
  }
template <class T>
void AdjLaunch<T>::recon(const Grid& g, int rc, int a, const T* W, const T* gWL, const T* gWR, T* S, T* gW,
                         const Fields<T, kPpmcRevFields>& X, cudaStream_t s) {
    if (rc == 0) recon_r<0>(g, a, W, gWL, gWR, S, gW, s);
    if (rc == 1) recon_r<1>(g, a, W, gWL, gWR, S, gW, s);
    if (rc == 2) {
      if constexpr (SplitPpmcRev<T>::v) {
        if (a == 0) launch_ppmc_rev<T, 0>(g, W, gWL, gWR, S, gW, X, s);
        if (a == 1) launch_ppmc_rev<T, 1>(g, W, gWL, gWR, S, gW, X, s);
        if (a == 2) launch_ppmc_rev<T, 2>(g, W, gWL, gWR, S, gW, X, s);
      } else {
        recon_r<2>(g, a, W, gWL, gWR, S, gW, s);
      }
    }
  }
template <class T>
void AdjLaunch<T>::prim(const Grid& g, bool half, const double* U, const double* Uh, const T* Bh, const T* gW, double* g5,
                   T* gBcc, cudaStream_t s) {
    if (half)
      k_adj_prim<T, true><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, U, Uh, Bh, gW, g5, gBcc);
    else
      k_adj_prim<T, false><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, U, Uh, Bh, gW, g5, gBcc);
  }
template <class T>
void AdjLaunch<T>::faces_n(const Grid& g, const double* g5, const T* gBcc, const T* gBf, double* gU, cudaStream_t s) {
    k_adj_faces_n<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, g5, gBcc, gBf, gU);
  }
template <class T>
void AdjLaunch<T>::fwd_half_keep(const Grid& g, const double* U, const T* F, const T* E, double dt, T* W, T* Bh, double* Uh,
                            cudaStream_t s) {
    k_fwd_half_keep<T><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, U, F, E, dt, W, Bh, Uh);
  }
template <class T>
void AdjLaunch<T>::hlld_batch(int n, double gamma, const double* wl, const double* wr, const double* bn, const double* gf,
                         double* gwl, double* gwr, double* gbn, double* f, cudaStream_t s) {
    k_hlld_vjp_batch<T><<<(n + 127) / 128, 128, 0, s>>>(n, gamma, wl, wr, bn, gf, gwl, gwr, gbn, f);
  }

}  // namespace mhd
