// mhd_adjoint.cuh -- hand-written reverse-mode derivatives of the step's
// local functions (HLLD, characteristic projections, PLMC, PPMC, primitive
// recovery).  Each *_vjp recomputes the forward function, follows the same
// branches (limiter selections, HLLD wave regions, degenerate-state switches,
// floors) and propagates the output cotangents back to the inputs.  Branch
// decisions carry no derivative.  Not in the paper: the adjoint of the
// VL+CT step is this library's addition; the forward functions are those of
// mhd_device.cuh (Sec. 2.2).
#pragma once

#include "mhd_device.cuh"

namespace mhd {

// ------------------------------------------------- forward-mode number --
// value + one directional derivative (the derivative of the CFL rate at one
// cell in the reverse of the dt reduction).
template <class T> struct Dl {
  T v, d;
  __device__ Dl() {}
  __device__ Dl(T x) : v(x), d(T(0)) {}
  __device__ Dl(T x, T dx) : v(x), d(dx) {}
};
template <class T> __device__ __forceinline__ Dl<T> operator+(Dl<T> a, Dl<T> b) { return Dl<T>(a.v + b.v, a.d + b.d); }
template <class T> __device__ __forceinline__ Dl<T> operator-(Dl<T> a, Dl<T> b) { return Dl<T>(a.v - b.v, a.d - b.d); }
template <class T> __device__ __forceinline__ Dl<T> operator-(Dl<T> a) { return Dl<T>(-a.v, -a.d); }
template <class T> __device__ __forceinline__ Dl<T> operator*(Dl<T> a, Dl<T> b) {
  return Dl<T>(a.v * b.v, a.d * b.v + a.v * b.d);
}
template <class T> __device__ __forceinline__ Dl<T> operator/(Dl<T> a, Dl<T> b) {
  const T q = a.v / b.v;
  return Dl<T>(q, (a.d - q * b.d) / b.v);
}
template <class T> __device__ __forceinline__ Dl<T> dsqrt(Dl<T> a) {
  const T s = tsqrt<T>(a.v);
  return Dl<T>(s, s > T(0) ? T(0.5) * a.d / s : T(0));
}

// cotangents of the eigen-system fields used by eig_left / eig_right
template <class T> struct EigG {
  T rho, ir, sr, isr, a, a2, ia2, af, as, cf, cs, Qf, Qs, Af, As, b1, b2;
  __device__ void zero() {
    rho = ir = sr = isr = a = a2 = ia2 = af = as = cf = cs = Qf = Qs = Af = As = b1 = b2 = T(0);
  }
};

// reverse of eig_left (q = L dw): accumulates gdw and gE
template <class T>
__device__ __forceinline__ void eig_left_vjp(const Eig<T>& E, T ir, const T* dw, const T* gq, T* gdw, EigG<T>& gE) {
  const T n = T(0.5) * E.ia2;
  const T bv = E.b1 * dw[2] + E.b2 * dw[3];
  const T bb0 = E.b1 * dw[5] + E.b2 * dw[6];
  const T bb = bb0 * E.isr;
  const T Xf = E.af * dw[4] * ir + E.as * E.a * bb;
  const T Yf = -E.af * E.cf * dw[1] + E.Qs * bv;
  const T Xs = E.as * dw[4] * ir - E.af * E.a * bb;
  const T Ys = -E.as * E.cs * dw[1] - E.Qf * bv;
  const T zb0 = -E.b2 * dw[5] + E.b1 * dw[6];
  const T gn = gq[0] * (Xf + Yf) + gq[2] * (Xs + Ys) + gq[4] * (Xs - Ys) + gq[6] * (Xf - Yf);
  const T gXf = n * (gq[0] + gq[6]), gYf = n * (gq[0] - gq[6]);
  const T gXs = n * (gq[2] + gq[4]), gYs = n * (gq[2] - gq[4]);
  const T gZ = gq[1] + gq[5], gZb = gq[1] - gq[5];
  gdw[0] += gq[3];
  gdw[4] += -gq[3] * E.ia2;
  gE.ia2 += -gq[3] * dw[4] + T(0.5) * gn;
  // Zb = 0.5 sg zb0 isr
  const T hz = T(0.5) * E.sg * gZb;
  gE.b2 += -hz * dw[5] * E.isr;
  gE.b1 += hz * dw[6] * E.isr;
  gdw[5] += -hz * E.b2 * E.isr;
  gdw[6] += hz * E.b1 * E.isr;
  gE.isr += hz * zb0;
  // Z = 0.5 (-b2 dw2 + b1 dw3)
  gE.b2 += -T(0.5) * gZ * dw[2];
  gE.b1 += T(0.5) * gZ * dw[3];
  gdw[2] += -T(0.5) * gZ * E.b2;
  gdw[3] += T(0.5) * gZ * E.b1;
  T gbv = T(0), gbb = T(0);
  // Ys = -as cs dw1 - Qf bv
  gE.as += -gYs * E.cs * dw[1];
  gE.cs += -gYs * E.as * dw[1];
  gdw[1] += -gYs * E.as * E.cs;
  gE.Qf += -gYs * bv;
  gbv += -gYs * E.Qf;
  // Xs = as dw4 ir - af a bb
  gE.as += gXs * dw[4] * ir;
  gdw[4] += gXs * E.as * ir;
  gE.ir += gXs * E.as * dw[4];
  gE.af += -gXs * E.a * bb;
  gE.a += -gXs * E.af * bb;
  gbb += -gXs * E.af * E.a;
  // Yf = -af cf dw1 + Qs bv
  gE.af += -gYf * E.cf * dw[1];
  gE.cf += -gYf * E.af * dw[1];
  gdw[1] += -gYf * E.af * E.cf;
  gE.Qs += gYf * bv;
  gbv += gYf * E.Qs;
  // Xf = af dw4 ir + as a bb
  gE.af += gXf * dw[4] * ir;
  gdw[4] += gXf * E.af * ir;
  gE.ir += gXf * E.af * dw[4];
  gE.as += gXf * E.a * bb;
  gE.a += gXf * E.as * bb;
  gbb += gXf * E.as * E.a;
  // bb = (b1 dw5 + b2 dw6) isr
  gE.b1 += gbb * dw[5] * E.isr;
  gE.b2 += gbb * dw[6] * E.isr;
  gdw[5] += gbb * E.b1 * E.isr;
  gdw[6] += gbb * E.b2 * E.isr;
  gE.isr += gbb * bb0;
  // bv = b1 dw2 + b2 dw3
  gE.b1 += gbv * dw[2];
  gE.b2 += gbv * dw[3];
  gdw[2] += gbv * E.b1;
  gdw[3] += gbv * E.b2;
}

// reverse of eig_right (dw = R q): accumulates gq and gE
template <class T>
__device__ __forceinline__ void eig_right_vjp(const Eig<T>& E, const T* q, const T* gdw, T* gq, EigG<T>& gE) {
  const T fp = q[0] + q[6], fm = q[0] - q[6];
  const T sp = q[2] + q[4], sm = q[2] - q[4];
  const T ap = q[1] + q[5], am = q[1] - q[5];
  const T cfa = E.cf * E.af, csa = E.cs * E.as;
  const T K = E.af * fp + E.as * sp;
  const T M = E.Qs * fm - E.Qf * sm;
  const T ms = E.As * fp - E.Af * sp;
  const T ssr = E.sg * E.sr * am;
  gE.b1 += gdw[5] * ms + gdw[6] * ssr + gdw[2] * M + gdw[3] * ap;
  gE.b2 += gdw[6] * ms - gdw[5] * ssr + gdw[3] * M - gdw[2] * ap;
  const T gms = gdw[5] * E.b1 + gdw[6] * E.b2;
  const T gssr = -gdw[5] * E.b2 + gdw[6] * E.b1;
  gE.sr += gssr * E.sg * am;
  T gam = gssr * E.sg * E.sr;
  gE.As += gms * fp;
  gE.Af += -gms * sp;
  T gfp = gms * E.As, gsp = -gms * E.Af;
  const T gK = gdw[0] * E.rho + gdw[4] * E.rho * E.a2;
  gE.rho += gdw[0] * K + gdw[4] * E.a2 * K;
  gE.a2 += gdw[4] * E.rho * K;
  const T gq3 = gdw[0];
  gE.af += gK * fp;
  gE.as += gK * sp;
  gfp += gK * E.af;
  gsp += gK * E.as;
  const T gM = gdw[2] * E.b1 + gdw[3] * E.b2;
  const T gap = -gdw[2] * E.b2 + gdw[3] * E.b1;
  gE.Qs += gM * fm;
  gE.Qf += -gM * sm;
  T gfm = gM * E.Qs, gsm = -gM * E.Qf;
  const T gcfa = -gdw[1] * fm, gcsa = -gdw[1] * sm;
  gfm += -gdw[1] * cfa;
  gsm += -gdw[1] * csa;
  gE.cf += gcfa * E.af;
  gE.af += gcfa * E.cf;
  gE.cs += gcsa * E.as;
  gE.as += gcsa * E.cs;
  gq[0] += gfp + gfm;
  gq[6] += gfp - gfm;
  gq[2] += gsp + gsm;
  gq[4] += gsp - gsm;
  gq[1] += gap + gam;
  gq[5] += gap - gam;
  gq[3] += gq3;
}

// Pushes the eigen-field cotangents back to (rho, P, B_t1, B_t2, B_n): one
// reverse sweep through the eigen-system formulas, written as plain roots
// and quotients (the forward eig_build folds them into reciprocal roots):
// ir = 1/rho, a2 = gamma P ir, ia2 = 1/a2, ca2 = B_n^2 ir, bt2 = |B_t|^2 ir,
// D = a2 - ca2 - bt2, sd = sqrt(D^2 + 4 a2 bt2), c_f^2 = (a2 + ca2 + bt2 + sd)/2,
// c_s^2 = a2 ca2 / c_f^2, the alpha pair sqrt((sd +- D)/(2 sd)) and
// sqrt(2 a2 bt2 / (sd (sd +- D))), beta = B_t/|B_t|, sqrt(rho), 1/sqrt(rho),
// a = sqrt(a2).  A root that is zero, and beta where |B_t|^2 < 1e-12 (B_n^2 +
// gamma P) (reading D-23), carry no derivative.
template <class T>
__device__ __forceinline__ void eig_fields_vjp(T gamma, const T* w0, T bn, const Eig<T>& E, const EigG<T>& gE,
                                               T* gw0, T& gbn) {
  const T rho = w0[0], p = w0[4], by = w0[5], bz = w0[6];
  // forward values: the roots and reciprocals come from the forward
  // eigensystem E of the same state (eig_build), the rest is recomputed
  const T ir = E.ir, a2 = E.a2, ia2 = E.ia2, cf = E.cf, cs = E.cs, sr = E.sr, isr = E.isr, a = E.a;
  const T ca2 = bn * bn * ir;
  const T bt2r = by * by + bz * bz;
  const T bt2 = bt2r * ir;
  const T b2 = ca2 + bt2;
  const T D = a2 - b2;
  const T sd = tsqrt<T>(D * D + T(4) * a2 * bt2);
  const T icf2 = E.rcf * E.rcf;
  const T cs2 = a2 * ca2 * icf2;
  const T sg = E.sg;
  // magnetosonic normalisations: af = sqrt(uf), as = sqrt(us)
  const int br = is0<T>(sd) ? 0 : (ge0<T>(D) ? 1 : 2);
  const T af = E.af, as = E.as;
  T M = T(0), N = T(0), iM = T(0), r2s = T(0);
  if (br != 0) {
    N = T(2) * a2 * bt2;
    M = br == 1 ? sd * (sd + D) : sd * (sd - D);
    iM = trcp<T>(M);
    r2s = trcp<T>(T(2) * sd);
  }
  const T ibt = gt0<T>(bt2r) ? trsqrt<T>(bt2r) : T(0);
  const bool bfree = gt0<T>(bt2r) && !(bt2r < T(1e-12) * (bn * bn + gamma * p));

  // reverse sweep
  T g_rho = gE.rho, g_ir = gE.ir, g_sr = gE.sr, g_isr = gE.isr, g_a = gE.a, g_a2 = gE.a2, g_ia2 = gE.ia2;
  T g_af = gE.af, g_as = gE.as, g_cf = gE.cf, g_cs = gE.cs;
  T g_by = T(0), g_bz = T(0), g_bn = T(0), g_p = T(0);
  // Qf = cf af sg, Qs = cs as sg, Af = a af sr, As = a as sr
  g_cf += gE.Qf * af * sg;
  g_af += gE.Qf * cf * sg;
  g_cs += gE.Qs * as * sg;
  g_as += gE.Qs * cs * sg;
  g_a += gE.Af * af * sr + gE.As * as * sr;
  g_af += gE.Af * a * sr;
  g_as += gE.As * a * sr;
  g_sr += gE.Af * a * af + gE.As * a * as;
  // a = sqrt(a2), isr = 1/sr, sr = sqrt(rho)
  if (a > T(0)) g_a2 += g_a * T(0.5) * (a * ia2);  // 1/a = a / a^2
  g_sr += -g_isr * isr * isr;
  if (sr > T(0)) g_rho += g_sr * T(0.5) * isr;
  // b1 = by / bt, b2 = bz / bt, bt = sqrt(bt2r)
  T g_bt2r = T(0);
  if (bfree) {
    g_by += gE.b1 * ibt;
    g_bz += gE.b2 * ibt;
    const T g_bt = -(gE.b1 * by + gE.b2 * bz) * ibt * ibt;
    g_bt2r += g_bt * T(0.5) * ibt;
  }
  // af, as
  T g_sd = T(0), g_D = T(0), g_bt2 = T(0);
  if (br != 0) {
    // big = (sd +- D) / (2 sd), small = N / M
    const T g_big = br == 1 ? (af > T(0) ? g_af * T(0.5) * trcp<T>(af) : T(0))
                            : (as > T(0) ? g_as * T(0.5) * trcp<T>(as) : T(0));
    const T g_small = br == 1 ? (as > T(0) ? g_as * T(0.5) * trcp<T>(as) : T(0))
                              : (af > T(0) ? g_af * T(0.5) * trcp<T>(af) : T(0));
    const T sD = br == 1 ? T(1) : T(-1);  // big = (sd + sD D) / (2 sd)
    // d big / d sd = -sD D / (2 sd^2), d big / d D = sD / (2 sd)
    g_sd += -g_big * sD * D * r2s * r2s * T(2);
    g_D += g_big * sD * r2s;
    const T g_N = g_small * iM;
    const T g_M = -g_small * N * iM * iM;
    g_a2 += g_N * T(2) * bt2;
    g_bt2 += g_N * T(2) * a2;
    // M = sd (sd + sD D)
    g_sd += g_M * (T(2) * sd + sD * D);
    g_D += g_M * sD * sd;
  }
  // cs = sqrt(cs2), cf = sqrt(cf2), cs2 = a2 ca2 / cf2, cf2 = (a2 + b2 + sd)/2
  T g_cs2 = cs > T(0) ? g_cs * T(0.5) * trcp<T>(cs) : T(0);
  T g_cf2 = cf > T(0) ? g_cf * T(0.5) * E.rcf : T(0);
  g_a2 += g_cs2 * ca2 * icf2;
  T g_ca2 = g_cs2 * a2 * icf2;
  g_cf2 += -g_cs2 * cs2 * icf2;
  g_a2 += T(0.5) * g_cf2;
  T g_b2 = T(0.5) * g_cf2;
  g_sd += T(0.5) * g_cf2;
  // sd = sqrt(D^2 + 4 a2 bt2)
  if (sd > T(0)) {
    const T g_X = g_sd * r2s;  // (sd > 0: r2s = 1/(2 sd))
    g_D += g_X * T(2) * D;
    g_a2 += g_X * T(4) * bt2;
    g_bt2 += g_X * T(4) * a2;
  }
  // D = a2 - b2, b2 = ca2 + bt2, bt2 = bt2r ir, bt2r = by^2 + bz^2, ca2 = bn^2 ir
  g_a2 += g_D;
  g_b2 += -g_D;
  g_ca2 += g_b2;
  g_bt2 += g_b2;
  g_bt2r += g_bt2 * ir;
  g_ir += g_bt2 * bt2r;
  g_by += g_bt2r * T(2) * by;
  g_bz += g_bt2r * T(2) * bz;
  g_bn += g_ca2 * T(2) * bn * ir;
  g_ir += g_ca2 * bn * bn;
  // ia2 = 1/a2, a2 = gamma p ir, ir = 1/rho
  g_a2 += -g_ia2 * ia2 * ia2;
  g_p += g_a2 * gamma * ir;
  g_ir += g_a2 * gamma * p;
  g_rho += -g_ir * ir * ir;
  gw0[0] += g_rho;
  gw0[4] += g_p;
  gw0[5] += g_by;
  gw0[6] += g_bz;
  gbn += g_bn;
}


// With every call inlined, the float-pair reverse reconstruction kernels
// outgrow the instruction cache (ncu: warps stalled mostly on instruction
// fetch; the PPMC kernels of y and z ran 3x slower than that of x).  For
// float pairs the per-field PPM limiter (forward and reverse), the
// projections and their reverses are calls: one copy each.
template <class T> struct OutlineRev { static constexpr bool v = false; };
template <> struct OutlineRev<df> { static constexpr bool v = true; };
template <class T> __device__ __noinline__ void ppm_one_call(const T* q, T& qm, T& qp) { ppm_one<T>(q, qm, qp); }
template <class T>
__device__ __noinline__ void eig_left_vjp_call(const Eig<T>& E, T ir, const T* dw, const T* gq, T* gdw, EigG<T>& gE) {
  eig_left_vjp<T>(E, ir, dw, gq, gdw, gE);
}
template <class T> __device__ __noinline__ void eig_left_call(const Eig<T>& E, const T* dw, T* q) { eig_left<T>(E, dw, q); }
template <class T>
__device__ __noinline__ void eig_right_vjp_call(const Eig<T>& E, const T* q, const T* gdw, T* gq, EigG<T>& gE) {
  eig_right_vjp<T>(E, q, gdw, gq, gE);
}
// the calls above where OutlineRev<T> holds, else the inlined functions
template <class T> __device__ __forceinline__ void eig_left_o(const Eig<T>& E, const T* dw, T* q) {
  if constexpr (OutlineRev<T>::v) eig_left_call<T>(E, dw, q);
  else eig_left<T>(E, dw, q);
}
template <class T>
__device__ __forceinline__ void eig_left_vjp_o(const Eig<T>& E, T ir, const T* dw, const T* gq, T* gdw, EigG<T>& gE) {
  if constexpr (OutlineRev<T>::v) eig_left_vjp_call<T>(E, ir, dw, gq, gdw, gE);
  else eig_left_vjp<T>(E, ir, dw, gq, gdw, gE);
}
template <class T>
__device__ __forceinline__ void eig_right_vjp_o(const Eig<T>& E, const T* q, const T* gdw, T* gq, EigG<T>& gE) {
  if constexpr (OutlineRev<T>::v) eig_right_vjp_call<T>(E, q, gdw, gq, gE);
  else eig_right_vjp<T>(E, q, gdw, gq, gE);
}

// ------------------------------------------------------------- PLMC VJP --
// gwl, gwr: cotangents of W_{L,i+1/2}, W_{R,i-1/2} (after the face floors).
// Accumulates into gwm, gw0, gwp (cells i-1, i, i+1) and gbn.
template <class T>
__device__ void plmc_vjp(T gamma, T rho_floor, T p_floor, const T* wm, const T* w0, const T* wp, T bn,
                         const T* gwl_in, const T* gwr_in, T* gwm, T* gw0, T* gwp, T& gbn) {
  T dL[7], dR[7], dG[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    dL[q] = w0[q] - wm[q];
    dR[q] = wp[q] - w0[q];
  }
  van_leer7<T>(dL, dR, dG);  // the forward's arithmetic (plmc)
  Eig<T> E;
  eig_build<T>(gamma, w0, bn, E);
  const T ir = E.ir;
  T aL[7], aR[7], aC[7], aG[7], am[7], dW[7];
  eig_left_o<T>(E, dL, aL);
  eig_left_o<T>(E, dR, aR);
  eig_left_o<T>(E, dG, aG);
#pragma unroll
  for (int q = 0; q < 7; ++q) aC[q] = T(0.5) * (aL[q] + aR[q]);
  int sel[7];  // -1: zero slope; 0..3: candidate 2|aL|, 2|aR|, |aC|, |aG|
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    sel[q] = -1;
    am[q] = T(0);
    if (pos_prod<T>(aL[q], aR[q])) {
      // the selections of the forward min_abs(min_abs(2 aL, 2 aR), min_abs(aC, aG)),
      // ties to the second operand
      const T c0 = fabs(twice<T>(aL[q])), c1 = fabs(twice<T>(aR[q])), c2 = fabs(aC[q]), c3 = fabs(aG[q]);
      const int s01 = nonneg_lt<T>(c0, c1) ? 0 : 1;
      const T m01 = s01 == 0 ? c0 : c1;
      const int s23 = nonneg_lt<T>(c2, c3) ? 2 : 3;
      const T m23 = s23 == 2 ? c2 : c3;
      const bool first = nonneg_lt<T>(m01, m23);
      sel[q] = first ? s01 : s23;
      am[q] = with_sign<T>(aC[q], first ? m01 : m23);
    }
  }
  eig_right<T>(E, am, dW);
  // faces with floors: cotangent passes where the floor did not bind
  T gwl[7], gwr[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    gwl[q] = gwl_in[q];
    gwr[q] = gwr_in[q];
  }
  if (w0[0] + T(0.5) * dW[0] < rho_floor) gwl[0] = T(0);
  if (w0[4] + T(0.5) * dW[4] < p_floor) gwl[4] = T(0);
  if (w0[0] - T(0.5) * dW[0] < rho_floor) gwr[0] = T(0);
  if (w0[4] - T(0.5) * dW[4] < p_floor) gwr[4] = T(0);
  T gdW[7], gam[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    gw0[q] += gwl[q] + gwr[q];
    gdW[q] = T(0.5) * (gwl[q] - gwr[q]);
    gam[q] = T(0);
  }
  EigG<T> gE;
  gE.zero();
  eig_right_vjp_o<T>(E, am, gdW, gam, gE);
  T gaL[7], gaR[7], gaC[7], gaG[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    gaL[q] = gaR[q] = gaC[q] = gaG[q] = T(0);
    if (sel[q] >= 0) {
      const T s = sgn0<T>(aC[q]) * gam[q];
      if (sel[q] == 0) gaL[q] = s * T(2) * sgn0<T>(aL[q]);
      if (sel[q] == 1) gaR[q] = s * T(2) * sgn0<T>(aR[q]);
      if (sel[q] == 2) gaC[q] = s * sgn0<T>(aC[q]);
      if (sel[q] == 3) gaG[q] = s * sgn0<T>(aG[q]);
    }
  }
  T gdL[7], gdR[7], gdG[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    gdL[q] = gdR[q] = gdG[q] = T(0);
    // aC = (aL + aR)/2
    gaL[q] += T(0.5) * gaC[q];
    gaR[q] += T(0.5) * gaC[q];
  }
  eig_left_vjp_o<T>(E, ir, dL, gaL, gdL, gE);
  eig_left_vjp_o<T>(E, ir, dR, gaR, gdR, gE);
  eig_left_vjp_o<T>(E, ir, dG, gaG, gdG, gE);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const T pr = dL[q] * dR[q];
    if (pr > T(0)) {
      // d dG/d dL = 2 (dR/s)^2, d dG/d dR = 2 (dL/s)^2 with s = dL + dR; the
      // ratios are bounded by 1, so nothing under- or overflows when s is tiny
      const T s = dL[q] + dR[q];
      const T is = trcp<T>(s);  // (dL dR > 0 without underflow: s is far from 0)
      const T rR = dR[q] * is, rL = dL[q] * is;
      gdL[q] += gdG[q] * T(2) * rR * rR;
      gdR[q] += gdG[q] * T(2) * rL * rL;
    }
    gwp[q] += gdR[q];
    gwm[q] += -gdL[q];
    gw0[q] += gdL[q] - gdR[q];
  }
  eig_fields_vjp<T>(gamma, w0, bn, E, gE, gw0, gbn);
}

// ------------------------------------------------------------- PPMC VJP --
// Reverse of ppm_one: q[0..4] deviations (q[2] = 0), cotangents gqm, gqp of
// the limited interface deviations; accumulates gq[0..4].
template <class T> __device__ __forceinline__ int d2sel3(T x, T y, T z) {
  // index of the limited value of d2lim3 (0: x, 1: C y, 2: C z), -1 for zero
  const T sx = sgn0<T>(x);
  if (!(sx != T(0) && sx == sgn0<T>(y) && sx == sgn0<T>(z))) return -1;
  const T a = fabs(x), b = T(1.25) * fabs(y), c = T(1.25) * fabs(z);
  // fmin(a, fmin(b, c))
  const int sbc = (c < b) ? 2 : 1;
  const T mbc = fmin(b, c);
  return (mbc < a) ? sbc : 0;
}
template <class T> __device__ __forceinline__ int d2sel4(T x, T y, T z, T t) {
  const T sx = sgn0<T>(x);
  if (!(sx != T(0) && sx == sgn0<T>(y) && sx == sgn0<T>(z) && sx == sgn0<T>(t))) return -1;
  const T a = fabs(x), b = T(1.25) * fabs(y), c = T(1.25) * fabs(z), d = T(1.25) * fabs(t);
  // fmin(fmin(a, b), fmin(c, d))
  const int sab = (b < a) ? 1 : 0;
  const T mab = fmin(a, b);
  const int scd = (d < c) ? 3 : 2;
  const T mcd = fmin(c, d);
  return (mcd < mab) ? scd : sab;
}

template <class T> __device__ void ppm_one_vjp(const T* q, T gqm, T gqp, T* gq) {
  const T c7 = from_d<T>(7.0 / 12.0), c1 = from_d<T>(1.0 / 12.0), c6 = from_d<T>(1.0 / 6.0);
  // forward, recording the branches
  T qm = c7 * (q[1] + q[2]) - c1 * (q[0] + q[3]);
  T qp = c7 * (q[2] + q[3]) - c1 * (q[1] + q[4]);
  const T d2m1 = q[0] - T(2) * q[1] + q[2];
  const T d20 = q[1] - T(2) * q[2] + q[3];
  const T d2p1 = q[2] - T(2) * q[3] + q[4];
  const bool limm = (qm - q[1]) * (q[2] - qm) < T(0);
  int sm_ = -1, sp_ = -1;
  if (limm) {
    const T d2c = T(3) * (q[1] - T(2) * qm + q[2]);
    sm_ = d2sel3<T>(d2c, d2m1, d20);
    qm = T(0.5) * (q[1] + q[2]) - d2lim3<T>(d2c, d2m1, d20) * c6;
  }
  const bool limp = (qp - q[2]) * (q[3] - qp) < T(0);
  if (limp) {
    const T d2c = T(3) * (q[2] - T(2) * qp + q[3]);
    sp_ = d2sel3<T>(d2c, d20, d2p1);
    qp = T(0.5) * (q[2] + q[3]) - d2lim3<T>(d2c, d20, d2p1) * c6;
  }
  const T dqm = q[2] - qm, dqp = qp - q[2];
  const bool ext = dqm * dqp <= T(0) || (q[2] - q[1]) * (q[3] - q[2]) <= T(0);
  // reverse of the cell limiter: cotangents of (qm, qp) after the interface limiter
  T g_qm = T(0), g_qp = T(0), g2m1 = T(0), g20 = T(0), g2p1 = T(0), gq2 = T(0);
  if (ext) {
    const T d2f = T(6) * (qm - T(2) * q[2] + qp);
    int s4 = -1;
    T r = T(0);
    if (d2f != T(0)) {
      s4 = d2sel4<T>(d2f, d2m1, d20, d2p1);
      r = d2lim4<T>(d2f, d2m1, d20, d2p1) / d2f;
    }
    // qm' = q2 - r dqm, qp' = q2 + r dqp
    const T gr = -gqm * dqm + gqp * dqp;
    const T gdqm = -gqm * r, gdqp = gqp * r;
    gq2 += gqm + gqp;
    // dqm = q2 - qm, dqp = qp - q2
    gq2 += gdqm - gdqp;
    g_qm += -gdqm;
    g_qp += gdqp;
    if (s4 > 0) {  // r = C d2_x / d2f; s4 == 0 gives r = 1 (constant)
      const T num = s4 == 1 ? d2m1 : (s4 == 2 ? d20 : d2p1);
      (void)num;
      const T gnum = gr * T(1.25) / d2f;
      // d r / d d2f = -r / d2f, written without squaring d2f (tiny in quiet regions)
      const T gd2f = -gr * r / d2f;
      if (s4 == 1) g2m1 += gnum;
      if (s4 == 2) g20 += gnum;
      if (s4 == 3) g2p1 += gnum;
      // d2f = 6 (qm - 2 q2 + qp)
      g_qm += T(6) * gd2f;
      g_qp += T(6) * gd2f;
      gq2 += -T(12) * gd2f;
    }
  } else {
    const bool clipm = fabs(dqm) >= T(2) * fabs(dqp);
    const bool clipp = fabs(dqp) >= T(2) * fabs(dqm);
    if (clipm) {  // qm' = q2 - 2 dqp = 3 q2 - 2 qp
      gq2 += T(3) * gqm;
      g_qp += -T(2) * gqm;
    } else {
      g_qm += gqm;
    }
    if (clipp) {  // qp' = q2 + 2 dqm = 3 q2 - 2 qm
      gq2 += T(3) * gqp;
      g_qm += -T(2) * gqp;
    } else {
      g_qp += gqp;
    }
  }
  // reverse of the interface limiter and the interpolation
  if (limm) {
    // qm = (q1 + q2)/2 - lim/6, lim in {d2c, C d2m1, C d20, 0}; d2c = 3 (q1 - 2 qm0 + q2)
    gq[1] += T(0.5) * g_qm;
    gq2 += T(0.5) * g_qm;
    const T gl = -g_qm * c6;
    if (sm_ == 0) {
      gq[1] += T(3) * gl;
      gq2 += T(3) * gl;
      const T gqm0 = -T(6) * gl;  // through the unlimited qm0
      gq[1] += c7 * gqm0;
      gq2 += c7 * gqm0;
      gq[0] += -c1 * gqm0;
      gq[3] += -c1 * gqm0;
    } else if (sm_ == 1) {
      g2m1 += T(1.25) * gl;
    } else if (sm_ == 2) {
      g20 += T(1.25) * gl;
    }
  } else {
    gq[1] += c7 * g_qm;
    gq2 += c7 * g_qm;
    gq[0] += -c1 * g_qm;
    gq[3] += -c1 * g_qm;
  }
  if (limp) {
    gq2 += T(0.5) * g_qp;
    gq[3] += T(0.5) * g_qp;
    const T gl = -g_qp * c6;
    if (sp_ == 0) {
      gq2 += T(3) * gl;
      gq[3] += T(3) * gl;
      const T gqp0 = -T(6) * gl;
      gq2 += c7 * gqp0;
      gq[3] += c7 * gqp0;
      gq[1] += -c1 * gqp0;
      gq[4] += -c1 * gqp0;
    } else if (sp_ == 1) {
      g20 += T(1.25) * gl;
    } else if (sp_ == 2) {
      g2p1 += T(1.25) * gl;
    }
  } else {
    gq2 += c7 * g_qp;
    gq[3] += c7 * g_qp;
    gq[1] += -c1 * g_qp;
    gq[4] += -c1 * g_qp;
  }
  // second differences
  gq[0] += g2m1;
  gq[1] += -T(2) * g2m1 + g20;
  gq2 += g2m1 - T(2) * g20 + g2p1;
  gq[3] += g20 - T(2) * g2p1;
  gq[4] += g2p1;
  gq[2] += gq2;
}

template <class T> __device__ __noinline__ void ppm_one_vjp_call(const T* q, T gqm, T gqp, T* gq) {
  ppm_one_vjp<T>(q, gqm, gqp, gq);
}

// Reverse of PPMC for one cell.  wload(m, w7) loads the directional state of
// stencil cell m (0..4 for i-2..i+2); put(m, g7) receives the cotangent of
// stencil cell m != 2, once each; gw2 (7) receives that of cell i and gbn
// that of its cell-centred B_n.  The stencil is loaded where it is used and
// the slots are written as they are formed, so the live state is the
// eigensystem, the characteristic deviations and their cotangents (holding
// the whole stencil and its cotangents spilled the float-pair kernel).
template <class T, class Load, class Put>
__device__ void ppmc_vjp(T gamma, T rho_floor, T p_floor, Load wload, T bn, const T* gwl_in, const T* gwr_in,
                         Put put, T* gw2, T& gbn) {
  T w2[7];
  wload(2, w2);
  Eig<T> E;
  eig_build<T>(gamma, w2, bn, E);
  const T ir = E.ir;
  T qs[4][7];  // deviations of cells i-2, i-1, i+1, i+2 (q of cell i is 0)
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T wm[7], d[7];
    wload(k < 2 ? k : k + 1, wm);
#pragma unroll
    for (int c = 0; c < 7; ++c) d[c] = wm[c] - w2[c];
    eig_left_o<T>(E, d, qs[k]);
  }
  T dm[7], dp[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    const T col[5] = {qs[0][c], qs[1][c], T(0), qs[2][c], qs[3][c]};
    T qm, qp;
    if constexpr (OutlineRev<T>::v) ppm_one_call<T>(col, qm, qp);
    else ppm_one<T>(col, qm, qp);
    dm[c] = qm;
    dp[c] = qp;
  }
  T Wm[7], Wp[7];
  eig_right<T>(E, dm, Wm);
  eig_right<T>(E, dp, Wp);
  T gwl[7], gwr[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    gwl[c] = gwl_in[c];
    gwr[c] = gwr_in[c];
  }
  if (w2[0] + Wp[0] < rho_floor) gwl[0] = T(0);
  if (w2[4] + Wp[4] < p_floor) gwl[4] = T(0);
  if (w2[0] + Wm[0] < rho_floor) gwr[0] = T(0);
  if (w2[4] + Wm[4] < p_floor) gwr[4] = T(0);
  EigG<T> gE;
  gE.zero();
  T gdm[7], gdp[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    gw2[c] = gwl[c] + gwr[c];
    gdm[c] = gdp[c] = T(0);
  }
  eig_right_vjp_o<T>(E, dp, gwl, gdp, gE);
  eig_right_vjp_o<T>(E, dm, gwr, gdm, gE);
  T gqs[4][7];
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    const T col[5] = {qs[0][c], qs[1][c], T(0), qs[2][c], qs[3][c]};
    T gcol[5] = {T(0), T(0), T(0), T(0), T(0)};
    if constexpr (OutlineRev<T>::v) ppm_one_vjp_call<T>(col, gdm[c], gdp[c], gcol);
    else ppm_one_vjp<T>(col, gdm[c], gdp[c], gcol);
    gqs[0][c] = gcol[0];
    gqs[1][c] = gcol[1];
    gqs[2][c] = gcol[3];
    gqs[3][c] = gcol[4];
    // gcol[2] is the cotangent of q_0, which is identically 0 (deviation form)
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T wm[7], d[7];
    wload(k < 2 ? k : k + 1, wm);
#pragma unroll
    for (int c = 0; c < 7; ++c) d[c] = wm[c] - w2[c];
    T gd[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    eig_left_vjp_o<T>(E, ir, d, gqs[k], gd, gE);
    put(k < 2 ? k : k + 1, gd);
#pragma unroll
    for (int c = 0; c < 7; ++c) gw2[c] -= gd[c];
  }
  eig_fields_vjp<T>(gamma, w2, bn, E, gE, gw2, gbn);
}


// The same reverse in three passes, for kernels that pass the intermediates
// through global memory (one-kernel form: the eigensystem, the 28
// characteristic deviations and their cotangents live at once; for float
// pairs that is 230 registers and a 1 KB stack frame per thread).  Every sum
// keeps the order of ppmc_vjp, so the three passes give its result bit for
// bit.
//   pass 1: forward reconstruction, face floors and the reverse of the
//           back-projections: gdm, gdp (7 each), gE, and gw2 = gwl + gwr;
//   pass 2: the deviations again and the reverse of the PPM limiter per
//           field: gq(k, 7) for the stencil cells k = 0, 1, 3, 4;
//   pass 3: the reverse of the projections (put(m, g7) per stencil cell m,
//           gw2 -= its cotangent) and of the eigensystem (gw2, gbn).
template <class T, class Load>
__device__ __forceinline__ void ppmc_deviations(T gamma, Load wload, T bn, T* w2, Eig<T>& E, T (*qs)[7]) {
  wload(2, w2);
  eig_build<T>(gamma, w2, bn, E);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T wm[7], d[7];
    wload(k < 2 ? k : k + 1, wm);
#pragma unroll
    for (int c = 0; c < 7; ++c) d[c] = wm[c] - w2[c];
    eig_left_o<T>(E, d, qs[k]);
  }
}

template <class T, class Load>
__device__ void ppmc_vjp_pass1(T gamma, T rho_floor, T p_floor, Load wload, T bn, const T* gwl_in, const T* gwr_in,
                               T* gdm, T* gdp, EigG<T>& gE, T* gw2) {
  T w2[7];
  Eig<T> E;
  T dm[7], dp[7];
  {
    T qs[4][7];
    ppmc_deviations<T>(gamma, wload, bn, w2, E, qs);
#pragma unroll
    for (int c = 0; c < 7; ++c) {
      const T col[5] = {qs[0][c], qs[1][c], T(0), qs[2][c], qs[3][c]};
      T qm, qp;
      if constexpr (OutlineRev<T>::v) ppm_one_call<T>(col, qm, qp);
      else ppm_one<T>(col, qm, qp);
      dm[c] = qm;
      dp[c] = qp;
    }
  }
  T Wm[7], Wp[7];
  eig_right<T>(E, dm, Wm);
  eig_right<T>(E, dp, Wp);
  T gwl[7], gwr[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    gwl[c] = gwl_in[c];
    gwr[c] = gwr_in[c];
  }
  if (w2[0] + Wp[0] < rho_floor) gwl[0] = T(0);
  if (w2[4] + Wp[4] < p_floor) gwl[4] = T(0);
  if (w2[0] + Wm[0] < rho_floor) gwr[0] = T(0);
  if (w2[4] + Wm[4] < p_floor) gwr[4] = T(0);
  gE.zero();
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    gw2[c] = gwl[c] + gwr[c];
    gdm[c] = gdp[c] = T(0);
  }
  eig_right_vjp_o<T>(E, dp, gwl, gdp, gE);
  eig_right_vjp_o<T>(E, dm, gwr, gdm, gE);
}

// gq[k][c]: cotangent of the deviation of stencil cell (0, 1, 3, 4)[k], field c
template <class T, class Load>
__device__ void ppmc_vjp_pass2(T gamma, Load wload, T bn, const T* gdm, const T* gdp, T (*gq)[7]) {
  T w2[7], qs[4][7];
  Eig<T> E;
  ppmc_deviations<T>(gamma, wload, bn, w2, E, qs);
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    const T col[5] = {qs[0][c], qs[1][c], T(0), qs[2][c], qs[3][c]};
    T gcol[5] = {T(0), T(0), T(0), T(0), T(0)};
    if constexpr (OutlineRev<T>::v) ppm_one_vjp_call<T>(col, gdm[c], gdp[c], gcol);
    else ppm_one_vjp<T>(col, gdm[c], gdp[c], gcol);
    gq[0][c] = gcol[0];
    gq[1][c] = gcol[1];
    gq[2][c] = gcol[3];
    gq[3][c] = gcol[4];
  }
}

// gqload(k, g7): the pass-2 cotangents of stencil cell (0, 1, 3, 4)[k]
template <class T, class Load, class GqLoad, class Put>
__device__ void ppmc_vjp_pass3(T gamma, Load wload, T bn, GqLoad gqload, EigG<T>& gE, T* gw2, Put put, T& gbn) {
  T w2[7];
  wload(2, w2);
  Eig<T> E;
  eig_build<T>(gamma, w2, bn, E);
  const T ir = E.ir;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    T wm[7], d[7], gq[7];
    wload(k < 2 ? k : k + 1, wm);
#pragma unroll
    for (int c = 0; c < 7; ++c) d[c] = wm[c] - w2[c];
    gqload(k, gq);
    T gd[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    eig_left_vjp_o<T>(E, ir, d, gq, gd, gE);
    put(k < 2 ? k : k + 1, gd);
#pragma unroll
    for (int c = 0; c < 7; ++c) gw2[c] -= gd[c];
  }
  eig_fields_vjp<T>(gamma, w2, bn, E, gE, gw2, gbn);
}

// the 17 eigensystem cotangents as an array (the pass-1 output)
template <class T> __device__ __forceinline__ void eigg_pack(const EigG<T>& e, T* v) {
  v[0] = e.rho; v[1] = e.ir; v[2] = e.sr; v[3] = e.isr; v[4] = e.a; v[5] = e.a2; v[6] = e.ia2; v[7] = e.af;
  v[8] = e.as; v[9] = e.cf; v[10] = e.cs; v[11] = e.Qf; v[12] = e.Qs; v[13] = e.Af; v[14] = e.As; v[15] = e.b1;
  v[16] = e.b2;
}
template <class T> __device__ __forceinline__ void eigg_unpack(const T* v, EigG<T>& e) {
  e.rho = v[0]; e.ir = v[1]; e.sr = v[2]; e.isr = v[3]; e.a = v[4]; e.a2 = v[5]; e.ia2 = v[6]; e.af = v[7];
  e.as = v[8]; e.cf = v[9]; e.cs = v[10]; e.Qf = v[11]; e.Qs = v[12]; e.Af = v[13]; e.As = v[14]; e.b1 = v[15];
  e.b2 = v[16];
}

// ------------------------------------------------------------- HLLD VJP --
// reverse of fast_speed: accumulates d c_f / d(rho, p, bl, bt1, bt2) * gcf
template <class T>
__device__ __forceinline__ void fast_speed_vjp(T gamma, T rho, T p, T bl, T bt1, T bt2, T gcf, T& grho, T& gp, T& gbl,
                                               T& gbt1, T& gbt2) {
  const T ir = trcp<T>(rho);
  const T a2 = gamma * p * ir;
  const T t2r = bt1 * bt1 + bt2 * bt2;
  const T t2 = t2r * ir;
  const T b2 = bl * bl * ir + t2;
  const T dd = a2 - b2;
  const T X = dd * dd + T(4) * a2 * t2;
  const T sX = tsqrt<T>(X);
  const T cf = tsqrt<T>(T(0.5) * (a2 + b2 + sX));
  if (!(cf > T(0))) return;
  const T gcf2 = gcf * T(0.5) * trcp<T>(cf);
  T ga2 = T(0.5) * gcf2, gb2 = T(0.5) * gcf2;
  const T gsX = T(0.5) * gcf2;
  T gt2 = T(0);
  if (sX > T(0)) {
    const T gX = gsX * T(0.5) * trcp<T>(sX);
    const T gdd = gX * T(2) * dd;
    ga2 += gX * T(4) * t2 + gdd;
    gt2 += gX * T(4) * a2;
    gb2 += -gdd;
  }
  gbl += gb2 * T(2) * bl * ir;
  T gir = gb2 * bl * bl;
  gt2 += gb2;
  gbt1 += gt2 * T(2) * bt1 * ir;
  gbt2 += gt2 * T(2) * bt2 * ir;
  gir += gt2 * t2r;
  gp += ga2 * gamma * ir;
  gir += ga2 * gamma * p;
  grho += -gir * ir * ir;
}

// reverse of the physical flux F(w) and conserved vector U(w) of one side:
// gF, gU cotangents; accumulates gw[7], gbn
template <class T>
__device__ __forceinline__ void phys_cons_vjp(T gm1i, const T* w, T bn, const T* gF, const T* gU, T* gw, T& gbn) {
  const T rho = w[0], u = w[1], v = w[2], ww = w[3], p = w[4], by = w[5], bz = w[6];
  const T bb = bn * bn + by * by + bz * bz;
  const T e = p * gm1i + T(0.5) * rho * (u * u + v * v + ww * ww) + T(0.5) * bb;
  const T pt = p + T(0.5) * bb;
  const T mu = rho * u;
  const T vb = u * bn + v * by + ww * bz;
  // F0 = mu; F1 = mu u + pt - bn^2; F2 = mu v - bn by; F3 = mu w - bn bz;
  // F4 = (e + pt) u - bn vb; F5 = by u - bn v; F6 = bz u - bn w
  T gmu = gF[0] + gF[1] * u + gF[2] * v + gF[3] * ww;
  T gu = gF[1] * mu + gF[4] * (e + pt) + gF[5] * by + gF[6] * bz;
  T gpt = gF[1] + gF[4] * u;
  T ge = gF[4] * u;
  T gv = gF[2] * mu - gF[5] * bn;
  T gww = gF[3] * mu - gF[6] * bn;
  T gby = -gF[2] * bn + gF[5] * u;
  T gbz = -gF[3] * bn + gF[6] * u;
  gbn += -T(2) * bn * gF[1] - gF[2] * by - gF[3] * bz - gF[4] * vb - gF[5] * v - gF[6] * ww;
  const T gvb = -gF[4] * bn;
  gu += gvb * bn;
  gbn += gvb * u;
  gv += gvb * by;
  gby += gvb * v;
  gww += gvb * bz;
  gbz += gvb * ww;
  T grho = gmu * u;
  gu += gmu * rho;
  // U = (rho, rho u, rho v, rho w, e, by, bz)
  grho += gU[0] + gU[1] * u + gU[2] * v + gU[3] * ww;
  gu += gU[1] * rho;
  gv += gU[2] * rho;
  gww += gU[3] * rho;
  ge += gU[4];
  gby += gU[5];
  gbz += gU[6];
  // e, pt
  T gp = ge * gm1i + gpt;
  grho += ge * T(0.5) * (u * u + v * v + ww * ww);
  gu += ge * rho * u;
  gv += ge * rho * v;
  gww += ge * rho * ww;
  const T gbb = T(0.5) * (ge + gpt);
  gbn += gbb * T(2) * bn;
  gby += gbb * T(2) * by;
  gbz += gbb * T(2) * bz;
  gw[0] += grho;
  gw[1] += gu;
  gw[2] += gv;
  gw[3] += gww;
  gw[4] += gp;
  gw[5] += gby;
  gw[6] += gbz;
}

// Reverse of hlld(): gf = cotangent of the 7 flux components; accumulates
// gwl[7], gwr[7] and gbn.  Follows the region selection, the degenerate
// switches and the outer-speed selections of the forward solver.
template <class T>
__device__ void hlld_vjp(T gamma, const T* wl, const T* wr, T bn, const T* gf, T* gwl, T* gwr, T& gbn) {
  const T bn2 = bn * bn;
  const T gm1i = trcp<T>(gamma - T(1));
  T eL, eR, ptL, ptR;
  {
    T bb = bn2 + wl[5] * wl[5] + wl[6] * wl[6];
    eL = wl[4] * gm1i + T(0.5) * wl[0] * (wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3]) + T(0.5) * bb;
    ptL = wl[4] + T(0.5) * bb;
    bb = bn2 + wr[5] * wr[5] + wr[6] * wr[6];
    eR = wr[4] * gm1i + T(0.5) * wr[0] * (wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3]) + T(0.5) * bb;
    ptR = wr[4] + T(0.5) * bb;
  }
  const T cfL = fast_speed<T>(gamma, wl[0], wl[4], bn, wl[5], wl[6]);
  const T cfR = fast_speed<T>(gamma, wr[0], wr[4], bn, wr[5], wr[6]);
  const T cmax = fmax(cfL, cfR);
  const bool cL = !(cfR > cfL);  // fmax(cfL, cfR) takes cfL on ties
  const T SL = fmin(wl[1], wr[1]) - cmax;
  const T SR = fmax(wl[1], wr[1]) + cmax;
  const T zero7[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
  if (SL >= T(0)) {
    phys_cons_vjp<T>(gm1i, wl, bn, gf, zero7, gwl, gbn);
    return;
  }
  if (SR <= T(0)) {
    phys_cons_vjp<T>(gm1i, wr, bn, gf, zero7, gwr, gbn);
    return;
  }
  const T uL = wl[1], uR = wr[1];
  const T dL = SL - uL, dR = SR - uR;
  const T rdL = wl[0] * dL, rdR = wr[0] * dR;
  const T den = rdR - rdL;
  const T iden = trcp<T>(den);
  const T numSM = rdR * uR - rdL * uL - ptR + ptL;
  const T SM = numSM * iden;
  const T numP = rdR * ptL - rdL * ptR + rdL * rdR * (uR - uL);
  const T pts = numP * iden;

  // star states of both sides (forward values)
  T Sv[2] = {SL, SR}, dv[2] = {dL, dR}, rdv[2] = {rdL, rdR}, ev[2] = {eL, eR}, ptv[2] = {ptL, ptR};
  const T* wv[2] = {wl, wr};
  T rs[2], vs[2], ws[2], bys[2], bzs[2], es[2], sq[2], rsq[2], iSMv[2], Dv[2], iDv[2], tv[2], qv[2], vbv[2], vbsv[2];
  bool degv[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T* w = wv[s];
    const T Sd = Sv[s] - SM;
    iSMv[s] = trcp<T>(Sd);
    rs[s] = rdv[s] * iSMv[s];
    Dv[s] = rdv[s] * Sd - bn2;
    degv[s] = fabs(Dv[s]) < Eps<T>::hlld * pts;
    if (degv[s]) {
      vs[s] = w[2];
      ws[s] = w[3];
      bys[s] = w[5];
      bzs[s] = w[6];
      iDv[s] = tv[s] = qv[s] = T(0);
    } else {
      iDv[s] = trcp<T>(Dv[s]);
      tv[s] = bn * (SM - w[1]) * iDv[s];
      vs[s] = w[2] - w[5] * tv[s];
      ws[s] = w[3] - w[6] * tv[s];
      qv[s] = (rdv[s] * dv[s] - bn2) * iDv[s];
      bys[s] = w[5] * qv[s];
      bzs[s] = w[6] * qv[s];
    }
    vbv[s] = w[1] * bn + w[2] * w[5] + w[3] * w[6];
    vbsv[s] = SM * bn + vs[s] * bys[s] + ws[s] * bzs[s];
    es[s] = (dv[s] * ev[s] - ptv[s] * w[1] + pts * SM + bn * (vbv[s] - vbsv[s])) * iSMv[s];
    // sqrt(rho*) and its reciprocal as the forward solver forms them
    rsq[s] = trsqrt<T>(rs[s]);
    sq[s] = rs[s] * rsq[s];
  }
  const bool dbl = !(T(0.5) * bn2 < Eps<T>::hlld * pts);
  T SsL = SM, SsR = SM, vss = 0, wss = 0, byss = 0, bzss = 0, vbss = 0, ess[2] = {0, 0}, inv = 0, sg = 0, abn = 0;
  if (dbl) {
    sg = bn > T(0) ? T(1) : T(-1);
    abn = fabs(bn);
    SsL = SM - abn * rsq[0];
    SsR = SM + abn * rsq[1];
    inv = trcp<T>(sq[0] + sq[1]);
    vss = (sq[0] * vs[0] + sq[1] * vs[1] + (bys[1] - bys[0]) * sg) * inv;
    wss = (sq[0] * ws[0] + sq[1] * ws[1] + (bzs[1] - bzs[0]) * sg) * inv;
    byss = (sq[0] * bys[1] + sq[1] * bys[0] + sq[0] * sq[1] * (vs[1] - vs[0]) * sg) * inv;
    bzss = (sq[0] * bzs[1] + sq[1] * bzs[0] + sq[0] * sq[1] * (ws[1] - ws[0]) * sg) * inv;
    vbss = SM * bn + vss * byss + wss * bzss;
    ess[0] = es[0] - sq[0] * (vbsv[0] - vbss) * sg;
    ess[1] = es[1] + sq[1] * (vbsv[1] - vbss) * sg;
  }
  const bool left = SM >= T(0);
  const int a = left ? 0 : 1;
  const T* w = wv[a];
  const T S = Sv[a];
  const T Ss = left ? SsL : SsR;
  const bool inner = dbl && (left ? (SsL < T(0)) : (SsR >= T(0)));
  const T U0[7] = {w[0], w[0] * w[1], w[0] * w[2], w[0] * w[3], ev[a], w[5], w[6]};
  const T Us[7] = {rs[a], rs[a] * SM, rs[a] * vs[a], rs[a] * ws[a], es[a], bys[a], bzs[a]};
  T Uss[7];
  if (inner) {
    Uss[0] = rs[a];
    Uss[1] = rs[a] * SM;
    Uss[2] = rs[a] * vss;
    Uss[3] = rs[a] * wss;
    Uss[4] = ess[a];
    Uss[5] = byss;
    Uss[6] = bzss;
  }

  // ---- reverse ----
  // f = F(w) - S U0 + (S - Ss) Us + Ss Uss   (inner)
  // f = F(w) - S U0 + S Us                    (otherwise)
  T gU0[7], gUs[7], gUss[7];
  T gS = T(0), gSs = T(0);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    gU0[q] = -S * gf[q];
    gUs[q] = (inner ? (S - Ss) : S) * gf[q];
    gUss[q] = inner ? Ss * gf[q] : T(0);
    gS += gf[q] * (Us[q] - U0[q]);
    if (inner) gSs += gf[q] * (Uss[q] - Us[q]);
  }
  // accumulators of the intermediate variables
  T gSM = T(0), gpts = T(0), gbn_loc = T(0);
  T grs[2] = {0, 0}, gvs[2] = {0, 0}, gws[2] = {0, 0}, gbys[2] = {0, 0}, gbzs[2] = {0, 0}, ges[2] = {0, 0},
    gsq[2] = {0, 0};
  T gvss = 0, gwss = 0, gbyss = 0, gbzss = 0, gvbss = 0, gess[2] = {0, 0}, ginv = 0;
  // physical flux and U0 of the selected side
  phys_cons_vjp<T>(gm1i, w, bn, gf, gU0, a == 0 ? gwl : gwr, gbn_loc);
  // Uss
  if (inner) {
    grs[a] += gUss[0] + gUss[1] * SM + gUss[2] * vss + gUss[3] * wss;
    gSM += gUss[1] * rs[a];
    gvss += gUss[2] * rs[a];
    gwss += gUss[3] * rs[a];
    gess[a] += gUss[4];
    gbyss += gUss[5];
    gbzss += gUss[6];
  }
  // Us
  grs[a] += gUs[0] + gUs[1] * SM + gUs[2] * vs[a] + gUs[3] * ws[a];
  gSM += gUs[1] * rs[a];
  gvs[a] += gUs[2] * rs[a];
  gws[a] += gUs[3] * rs[a];
  ges[a] += gUs[4];
  gbys[a] += gUs[5];
  gbzs[a] += gUs[6];
  // S (outer speed of the selected side) and Ss
  T gSv[2] = {0, 0};
  gSv[a] += gS;
  if (dbl) {
    if (inner) {
      if (left) {  // SsL = SM - abn/sqL
        gSM += gSs;
        gsq[0] += gSs * abn * rsq[0] * rsq[0];
        gbn_loc += -gSs * sg * rsq[0];
      } else {  // SsR = SM + abn/sqR
        gSM += gSs;
        gsq[1] += -gSs * abn * rsq[1] * rsq[1];
        gbn_loc += gSs * sg * rsq[1];
      }
    }
    // ess_L = es_L - sqL (vbs_L - vbss) sg ; ess_R = es_R + sqR (vbs_R - vbss) sg
    T gvbs[2] = {0, 0};
    ges[0] += gess[0];
    gsq[0] += -gess[0] * (vbsv[0] - vbss) * sg;
    gvbs[0] += -gess[0] * sq[0] * sg;
    gvbss += gess[0] * sq[0] * sg;
    ges[1] += gess[1];
    gsq[1] += gess[1] * (vbsv[1] - vbss) * sg;
    gvbs[1] += gess[1] * sq[1] * sg;
    gvbss += -gess[1] * sq[1] * sg;
    // vbss = SM bn + vss byss + wss bzss
    gSM += gvbss * bn;
    gbn_loc += gvbss * SM;
    gvss += gvbss * byss;
    gbyss += gvbss * vss;
    gwss += gvbss * bzss;
    gbzss += gvbss * wss;
    // byss = Nby inv
    {
      const T N = sq[0] * bys[1] + sq[1] * bys[0] + sq[0] * sq[1] * (vs[1] - vs[0]) * sg;
      const T gN = gbyss * inv;
      ginv += gbyss * N;
      gsq[0] += gN * (bys[1] + sq[1] * (vs[1] - vs[0]) * sg);
      gsq[1] += gN * (bys[0] + sq[0] * (vs[1] - vs[0]) * sg);
      gbys[1] += gN * sq[0];
      gbys[0] += gN * sq[1];
      gvs[1] += gN * sq[0] * sq[1] * sg;
      gvs[0] += -gN * sq[0] * sq[1] * sg;
    }
    {
      const T N = sq[0] * bzs[1] + sq[1] * bzs[0] + sq[0] * sq[1] * (ws[1] - ws[0]) * sg;
      const T gN = gbzss * inv;
      ginv += gbzss * N;
      gsq[0] += gN * (bzs[1] + sq[1] * (ws[1] - ws[0]) * sg);
      gsq[1] += gN * (bzs[0] + sq[0] * (ws[1] - ws[0]) * sg);
      gbzs[1] += gN * sq[0];
      gbzs[0] += gN * sq[1];
      gws[1] += gN * sq[0] * sq[1] * sg;
      gws[0] += -gN * sq[0] * sq[1] * sg;
    }
    {
      const T N = sq[0] * vs[0] + sq[1] * vs[1] + (bys[1] - bys[0]) * sg;
      const T gN = gvss * inv;
      ginv += gvss * N;
      gsq[0] += gN * vs[0];
      gsq[1] += gN * vs[1];
      gvs[0] += gN * sq[0];
      gvs[1] += gN * sq[1];
      gbys[1] += gN * sg;
      gbys[0] += -gN * sg;
    }
    {
      const T N = sq[0] * ws[0] + sq[1] * ws[1] + (bzs[1] - bzs[0]) * sg;
      const T gN = gwss * inv;
      ginv += gwss * N;
      gsq[0] += gN * ws[0];
      gsq[1] += gN * ws[1];
      gws[0] += gN * sq[0];
      gws[1] += gN * sq[1];
      gbzs[1] += gN * sg;
      gbzs[0] += -gN * sg;
    }
    // inv = 1/(sqL + sqR)
    gsq[0] += -ginv * inv * inv;
    gsq[1] += -ginv * inv * inv;
    // the vbs cotangents join the star-state reverse below
    // (stored back into the per-side accumulators)
    T* gw2[2] = {gwl, gwr};
    (void)gw2;
    // vbs_s = SM bn + vs bys + ws bzs
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      gSM += gvbs[s] * bn;
      gbn_loc += gvbs[s] * SM;
      gvs[s] += gvbs[s] * bys[s];
      gbys[s] += gvbs[s] * vs[s];
      gws[s] += gvbs[s] * bzs[s];
      gbzs[s] += gvbs[s] * ws[s];
    }
  }
  // single-star states, both sides
  T grd[2] = {0, 0}, gd[2] = {0, 0}, ge[2] = {0, 0}, gpt[2] = {0, 0};
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T* ws_in = wv[s];
    T* gw = s == 0 ? gwl : gwr;
    // sq = sqrt(rs)
    if (sq[s] > T(0)) grs[s] += gsq[s] * T(0.5) * rsq[s];
    // es = Ne iSM, Ne = d e - pt u + pts SM + bn (vb - vbs)
    const T Ne = dv[s] * ev[s] - ptv[s] * ws_in[1] + pts * SM + bn * (vbv[s] - vbsv[s]);
    const T gNe = ges[s] * iSMv[s];
    T giSM = ges[s] * Ne;
    gd[s] += gNe * ev[s];
    ge[s] += gNe * dv[s];
    gpt[s] += -gNe * ws_in[1];
    gw[1] += -gNe * ptv[s];
    gpts += gNe * SM;
    gSM += gNe * pts;
    gbn_loc += gNe * (vbv[s] - vbsv[s]);
    const T gvb = gNe * bn;
    const T gvbs = -gNe * bn;
    // vbs = SM bn + vs bys + ws bzs
    gSM += gvbs * bn;
    gbn_loc += gvbs * SM;
    gvs[s] += gvbs * bys[s];
    gbys[s] += gvbs * vs[s];
    gws[s] += gvbs * bzs[s];
    gbzs[s] += gvbs * ws[s];
    // vb = u bn + v by + w bz
    gw[1] += gvb * bn;
    gbn_loc += gvb * ws_in[1];
    gw[2] += gvb * ws_in[5];
    gw[5] += gvb * ws_in[2];
    gw[3] += gvb * ws_in[6];
    gw[6] += gvb * ws_in[3];
    T gD = T(0);
    if (degv[s]) {
      gw[2] += gvs[s];
      gw[3] += gws[s];
      gw[5] += gbys[s];
      gw[6] += gbzs[s];
    } else {
      // bys = by q, bzs = bz q
      gw[5] += gbys[s] * qv[s];
      gw[6] += gbzs[s] * qv[s];
      const T gq = gbys[s] * ws_in[5] + gbzs[s] * ws_in[6];
      // q = (rd d - bn2) iD
      const T gNq = gq * iDv[s];
      T giD = gq * (rdv[s] * dv[s] - bn2);
      grd[s] += gNq * dv[s];
      gd[s] += gNq * rdv[s];
      gbn_loc += -gNq * T(2) * bn;
      // vs = v - by t ; ws = w - bz t
      gw[2] += gvs[s];
      gw[3] += gws[s];
      gw[5] += -gvs[s] * tv[s];
      gw[6] += -gws[s] * tv[s];
      const T gt = -gvs[s] * ws_in[5] - gws[s] * ws_in[6];
      // t = bn (SM - u) iD
      gbn_loc += gt * (SM - ws_in[1]) * iDv[s];
      gSM += gt * bn * iDv[s];
      gw[1] += -gt * bn * iDv[s];
      giD += gt * bn * (SM - ws_in[1]);
      gD += -giD * iDv[s] * iDv[s];
    }
    // D = rd Sd - bn2, Sd = S - SM
    const T Sd = Sv[s] - SM;
    grd[s] += gD * Sd;
    T gSd = gD * rdv[s];
    gbn_loc += -gD * T(2) * bn;
    // rs = rd iSM
    grd[s] += grs[s] * iSMv[s];
    giSM += grs[s] * rdv[s];
    gSd += -giSM * iSMv[s] * iSMv[s];
    gSv[s] += gSd;
    gSM += -gSd;
  }
  // middle wave: pts = numP iden, SM = numSM iden
  const T gnumP = gpts * iden;
  T giden = gpts * numP + gSM * numSM;
  const T gnumSM = gSM * iden;
  grd[1] += gnumP * (ptL + rdL * (uR - uL));
  gpt[0] += gnumP * rdR;
  grd[0] += gnumP * (-ptR + rdR * (uR - uL));
  gpt[1] += -gnumP * rdL;
  gwr[1] += gnumP * rdL * rdR;
  gwl[1] += -gnumP * rdL * rdR;
  grd[1] += gnumSM * uR;
  gwr[1] += gnumSM * rdR;
  grd[0] += -gnumSM * uL;
  gwl[1] += -gnumSM * rdL;
  gpt[1] += -gnumSM;
  gpt[0] += gnumSM;
  const T gden = -giden * iden * iden;
  grd[1] += gden;
  grd[0] += -gden;
  // rd = rho d ; d = S - u
  gwl[0] += grd[0] * dL;
  gd[0] += grd[0] * wl[0];
  gwr[0] += grd[1] * dR;
  gd[1] += grd[1] * wr[0];
  gSv[0] += gd[0];
  gwl[1] += -gd[0];
  gSv[1] += gd[1];
  gwr[1] += -gd[1];
  // e, pt of both sides (the star energies use them)
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T* ws_in = wv[s];
    T* gw = s == 0 ? gwl : gwr;
    gw[4] += ge[s] * gm1i + gpt[s];
    gw[0] += ge[s] * T(0.5) * (ws_in[1] * ws_in[1] + ws_in[2] * ws_in[2] + ws_in[3] * ws_in[3]);
    gw[1] += ge[s] * ws_in[0] * ws_in[1];
    gw[2] += ge[s] * ws_in[0] * ws_in[2];
    gw[3] += ge[s] * ws_in[0] * ws_in[3];
    const T gbb = T(0.5) * (ge[s] + gpt[s]);
    gbn_loc += gbb * T(2) * bn;
    gw[5] += gbb * T(2) * ws_in[5];
    gw[6] += gbb * T(2) * ws_in[6];
  }
  // outer speeds: SL = min(uL, uR) - cmax, SR = max(uL, uR) + cmax
  const T gcmax = -gSv[0] + gSv[1];
  if (wl[1] <= wr[1]) gwl[1] += gSv[0];
  else gwr[1] += gSv[0];
  if (wl[1] >= wr[1]) gwl[1] += gSv[1];
  else gwr[1] += gSv[1];
  if (cL)
    fast_speed_vjp<T>(gamma, wl[0], wl[4], bn, wl[5], wl[6], gcmax, gwl[0], gwl[4], gbn_loc, gwl[5], gwl[6]);
  else
    fast_speed_vjp<T>(gamma, wr[0], wr[4], bn, wr[5], wr[6], gcmax, gwr[0], gwr[4], gbn_loc, gwr[5], gwr[6]);
  gbn += gbn_loc;
}

// ------------------------------------------------- primitive recovery VJP --
// W = (rho', v, P', B_cc) from (rho, m, E, B_cc) as in prim_core; gW[8]
// cotangents; returns g of (rho, m0, m1, m2, E) in g5 and adds to gb[3].
__device__ __forceinline__ void prim_vjp(const Grid& g, double r, double m0, double m1, double m2, double e,
                                         const double* b, const double* gW, double* g5, double* gb) {
  const bool rfl = !(r >= g.rho_floor);  // fmax(r, floor) takes the floor
  const double rho = fmax(r, g.rho_floor);
  const double ir = __drcp_rn(rho);  // (the correctly rounded 1/rho)
  const double v0 = m0 * ir, v1 = m1 * ir, v2 = m2 * ir;
  const double ke = 0.5 * (m0 * v0 + m1 * v1 + m2 * v2);
  const double me = 0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
  const double p = (g.gamma - 1.0) * (e - ke - me);
  const bool pfl = !(p >= g.p_floor);
  const double gP = pfl ? 0.0 : gW[4];
  double grho = gW[0];
  double gv0 = gW[1], gv1 = gW[2], gv2 = gW[3];
  const double ge = (g.gamma - 1.0) * gP;
  const double gke = -ge, gme = -ge;
  gb[0] += gW[5] + gme * b[0];
  gb[1] += gW[6] + gme * b[1];
  gb[2] += gW[7] + gme * b[2];
  double gm0 = 0.5 * gke * v0, gm1 = 0.5 * gke * v1, gm2 = 0.5 * gke * v2;
  gv0 += 0.5 * gke * m0;
  gv1 += 0.5 * gke * m1;
  gv2 += 0.5 * gke * m2;
  gm0 += gv0 * ir;
  gm1 += gv1 * ir;
  gm2 += gv2 * ir;
  const double gir = gv0 * m0 + gv1 * m1 + gv2 * m2;
  grho += -gir * ir * ir;
  g5[0] = rfl ? 0.0 : grho;
  g5[1] = gm0;
  g5[2] = gm1;
  g5[3] = gm2;
  g5[4] = ge;
}

// The same reverse for the FP32-bulk mode: the floor decisions from the
// double pressure recovery as the FP32-bulk forward forms it
// (P = (gamma - 1)(E - (|m|^2 / rho' + |B_cc|^2) / 2)), the derivative
// arithmetic in float; gb[3] is written, not accumulated.
__device__ __forceinline__ void prim_vjp_f32(const Grid& g, double r, double m0, double m1, double m2, double e,
                                             const double* b, const float* gW, float* g5, float* gb) {
  const bool rfl = !(r >= g.rho_floor);
  const double rho = fmax(r, g.rho_floor);
  const double ir = __drcp_rn(rho);
  const double kem = 0.5 * ((m0 * m0 + m1 * m1 + m2 * m2) * ir + (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]));
  const bool pfl = !(g.gm1 * (e - kem) >= g.p_floor);
  const float irf = d2f_bits(ir), gm1 = d2f_bits(g.gm1);
  const float m[3] = {d2f_bits(m0), d2f_bits(m1), d2f_bits(m2)};
  const float bf[3] = {d2f_bits(b[0]), d2f_bits(b[1]), d2f_bits(b[2])};
  const float ge = pfl ? 0.0f : gm1 * gW[4];
  // ke = |m|^2 / (2 rho'), me = |B_cc|^2 / 2, both entering P with -ge
  float gir = 0.0f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float v = m[a] * irf;
    gb[a] = gW[5 + a] - ge * bf[a];
    // v = m ir: gm += gv ir, gir += gv m; ke: gm += -ge v
    g5[1 + a] = gW[1 + a] * irf - ge * v;
    gir += gW[1 + a] * m[a];
  }
  // d ke / d ir = |m|^2 / 2: gir += -ge |m|^2 / 2
  gir += -0.5f * ge * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  const float grho = gW[0] - gir * irf * irf;
  g5[0] = rfl ? 0.0f : grho;
  g5[4] = ge;
}

}  // namespace mhd
