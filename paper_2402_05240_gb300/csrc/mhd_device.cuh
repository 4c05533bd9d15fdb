// mhd_device.cuh -- device arithmetic of the VL+CT ideal-MHD step (sm_103a).
//
// Templated on the compute type T (double for the FP64 step, float for the
// FP32-bulk step).  Pressure recovery from the conserved state is always done
// in double (the cancellation E - KE - B^2/2 sets the pressure floor).
//
// Method: Caddy & Schneider (arXiv:2402.05240) Sec. 2.1-2.2; HLLD of Miyoshi
// & Kusano (2005); primitive eigenvectors in the normalisation of Stone et
// al. (2008, App. A) with the left eigenvectors in closed form; PPM limiters
// of Colella & Sekora (2008) and McCorquodale & Colella (2011) applied in the
// characteristic variables (Felker & Stone 2018).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mhd_df.cuh"
#include "mhd_launch.h"

namespace mhd {

// ------------------------------------------------------------ grid helpers --
__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ long long cidx(const Grid& g, int i, int j, int k) {
  return ((long long)k * g.n[1] + j) * g.n[0] + i;
}

// index of cell (i,j,k) + s e_a, |s| < n[a]
template <int A>
__device__ __forceinline__ long long nb(const Grid& g, int i, int j, int k, int s) {
  if (A == 0) return cidx(g, wrapi(i + s, g.n[0]), j, k);
  if (A == 1) return cidx(g, i, wrapi(j + s, g.n[1]), k);
  return cidx(g, i, j, wrapi(k + s, g.n[2]));
}

template <class T> __device__ __forceinline__ T tsqrt(T x);
template <> __device__ __forceinline__ double tsqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float tsqrt<float>(float x) { return sqrtf(x); }

// correctly rounded reciprocal (cheaper than a general division) and the
// library reciprocal square root
template <class T> __device__ __forceinline__ T trcp(T x);
template <> __device__ __forceinline__ double trcp<double>(double x) { return __drcp_rn(x); }
template <> __device__ __forceinline__ float trcp<float>(float x) { return __frcp_rn(x); }
template <class T> __device__ __forceinline__ T trsqrt(T x);
template <> __device__ __forceinline__ double trsqrt<double>(double x) { return rsqrt(x); }
template <> __device__ __forceinline__ float trsqrt<float>(float x) { return rsqrtf(x); }

template <> __device__ __forceinline__ df tsqrt<df>(df x) { return df_sqrt(x); }
template <> __device__ __forceinline__ df trcp<df>(df x) { return df(1.0f, 0.0f) / x; }
template <> __device__ __forceinline__ df trsqrt<df>(df x) { return df_rsqrt(x); }

// Comparisons of the step's branch decisions.  The generic forms use
// floating-point compares; for double they test the bit pattern on the
// integer pipes (the FP64 pipe bounds the FP64 step), with the same result
// for every non-NaN operand.  Positive doubles order like their bit
// patterns as signed 64-bit integers; -0 is the most negative pattern.
constexpr long long kAbsBits = 0x7fffffffffffffffLL;
constexpr long long kNegZero = (long long)0x8000000000000000ULL;
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
template <class T> __device__ __forceinline__ bool ge0(T x) { return x >= T(0); }
template <class T> __device__ __forceinline__ bool gt0(T x) { return x > T(0); }
template <class T> __device__ __forceinline__ bool lt0(T x) { return x < T(0); }
template <class T> __device__ __forceinline__ bool le0(T x) { return x <= T(0); }
template <class T> __device__ __forceinline__ bool is0(T x) { return x == T(0); }
// |x| < t for t >= 0
template <class T> __device__ __forceinline__ bool abs_lt(T x, T t) { return fabs(x) < t; }
// x < t for x, t >= 0
template <class T> __device__ __forceinline__ bool nonneg_lt(T x, T t) { return x < t; }
// x < t for t > 0 (x of any sign)
template <class T> __device__ __forceinline__ bool lt_pos(T x, T t) { return x < t; }
// max(x, t) for t > 0 (x of any sign)
template <class T> __device__ __forceinline__ T max_pos(T x, T t) { return fmax(x, t); }
// max(x, y) for x, y >= 0
template <class T> __device__ __forceinline__ T max_nonneg(T x, T y) { return fmax(x, y); }
// min and max of two values of any sign
template <class T> __device__ __forceinline__ T min_s(T x, T y) { return fmin(x, y); }
template <class T> __device__ __forceinline__ T max_s(T x, T y) { return fmax(x, y); }

template <> __device__ __forceinline__ bool ge0<double>(double x) {
  const long long b = dbits(x);
  return (b >= 0) | (b == kNegZero);
}
template <> __device__ __forceinline__ bool gt0<double>(double x) { return dbits(x) > 0; }
template <> __device__ __forceinline__ bool lt0<double>(double x) {
  const long long b = dbits(x);
  return (b < 0) & (b != kNegZero);
}
template <> __device__ __forceinline__ bool le0<double>(double x) { return dbits(x) <= 0; }
template <> __device__ __forceinline__ bool is0<double>(double x) { return (dbits(x) & kAbsBits) == 0; }
template <> __device__ __forceinline__ bool abs_lt<double>(double x, double t) {
  return (dbits(x) & kAbsBits) < dbits(t);
}
template <> __device__ __forceinline__ bool nonneg_lt<double>(double x, double t) { return dbits(x) < dbits(t); }
template <> __device__ __forceinline__ bool lt_pos<double>(double x, double t) { return dbits(x) < dbits(t); }
template <> __device__ __forceinline__ double max_pos<double>(double x, double t) {
  return dbits(x) > dbits(t) ? x : t;
}
template <> __device__ __forceinline__ double max_nonneg<double>(double x, double y) {
  return dbits(x) >= dbits(y) ? x : y;
}
// x finite (not +-inf, not NaN), and x > 0 and not NaN, on the bit pattern
__device__ __forceinline__ bool finite_bits(double x) { return (dbits(x) & kAbsBits) < 0x7ff0000000000000LL; }
__device__ __forceinline__ bool pos_bits(double x) {
  const long long b = dbits(x);
  return b > 0 && b <= 0x7ff0000000000000LL;
}
// |x|; for double on the bit pattern
template <class T> __device__ __forceinline__ T absv(T x) { return fabs(x); }
template <> __device__ __forceinline__ double absv<double>(double x) { return __longlong_as_double(dbits(x) & kAbsBits); }
// order key: sign-magnitude patterns mapped to a monotone signed integer
__device__ __forceinline__ long long dkey(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & kAbsBits);
}
template <> __device__ __forceinline__ double min_s<double>(double x, double y) {
  return dkey(y) < dkey(x) ? y : x;
}
template <> __device__ __forceinline__ double max_s<double>(double x, double y) {
  return dkey(x) < dkey(y) ? y : x;
}

// Conversions between the compute type and double without the conversion
// instructions, which issue at the FP64 rate on this GPU (mhd_df.cuh).
template <class T> __device__ __forceinline__ double to_d(T x);
template <> __device__ __forceinline__ double to_d<double>(double x) { return x; }
template <> __device__ __forceinline__ double to_d<float>(float x) { return f2d_bits(x); }
template <> __device__ __forceinline__ double to_d<df>(df x) { return (double)x; }
template <class T> __device__ __forceinline__ T from_d(double x);
template <> __device__ __forceinline__ double from_d<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_d<float>(double x) { return d2f_bits(x); }
template <> __device__ __forceinline__ df from_d<df>(double x) { return df(x); }

// Exact<T>: the full update widens each flux and edge value to double before
// differencing (a difference of two floats is exact in double).  df values
// already carry ~48 bits, so their differences and increments are formed in
// df and added to the double state once.
template <class T> struct Exact { static constexpr bool full = true; };
template <> struct Exact<df> { static constexpr bool full = false; };

template <class T> struct Eps;
template <> struct Eps<double> { static constexpr double hlld = 1e-8; };
template <> struct Eps<float> { static constexpr float hlld = 1e-4f; };
template <> struct Eps<df> { static constexpr float hlld = 1e-8f; };

// ------------------------------------------------- primitives (Sec. 2.2.1) --
// Cell primitives: rho, v, P (pressure recovered in double) and B_cc, the mean
// of the two faces of each component.
struct PrimD {
  double rho, v[3], p, b[3];
};

// ----------------------------------------------------- fast speed (Eq. c_f) --
// c_f^2 = (a2 + b2 + sqrt((a2 - b2)^2 + 4 a2 bt2)) / 2 with a2 = gamma P / rho,
// b2 = |B|^2 / rho, bt2 = |B_t|^2 / rho: the printed discriminant
// (gamma P + B^2)^2 - 4 gamma P B_l^2 (over rho^2) as a sum of non-negative terms.
template <class T>
__device__ __forceinline__ T fast_speed_sq(T gamma, T rho, T p, T bl, T bt1, T bt2) {
  T ir = trcp<T>(rho);
  T a2 = gamma * p * ir;
  T t2 = (bt1 * bt1 + bt2 * bt2) * ir;
  T b2 = bl * bl * ir + t2;
  T dd = a2 - b2;
  return T(0.5) * (a2 + b2 + tsqrt<T>(dd * dd + T(4) * a2 * t2));
}
template <class T>
__device__ __forceinline__ T fast_speed(T gamma, T rho, T p, T bl, T bt1, T bt2) {
  return tsqrt<T>(fast_speed_sq<T>(gamma, rho, p, bl, bt1, bt2));
}

// ------------------------------------------------------------------- HLLD --
// Miyoshi & Kusano (2005) in the solver frame; w = (rho, u, v, w, P, By, Bz),
// bn = longitudinal face field.  Outer speeds S_L = min(u) - max(c_f),
// S_R = max(u) + max(c_f); degenerate star / double-star states below
// Eps<T>::hlld * p_T*; flux selection with ties to the left.  gm1i = 1/(gamma - 1).
template <class T>
__device__ __forceinline__ void hlld(T gamma, T gm1i, const T* wl, const T* wr, T bn, T* f) {
  const T bn2 = bn * bn;
  // total pressures of both sides; the conserved energy is formed only for
  // the side whose states the flux is taken from
  const T btL = wl[5] * wl[5] + wl[6] * wl[6], btR = wr[5] * wr[5] + wr[6] * wr[6];
  const T bbL = bn2 + btL;
  const T bbR = bn2 + btR;
  const T ptL = wl[4] + T(0.5) * bbL;
  const T ptR = wr[4] + T(0.5) * bbR;
  auto energy = [&](const T* w, T bb) {
    return w[4] * gm1i + T(0.5) * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]) + T(0.5) * bb;
  };
  // max(c_f,L, c_f,R) (Eq. c_f with the face B_n): rho c_f^2 =
  // (gamma P + B^2 + sqrt((gamma P - B^2)^2 + 4 gamma P B_t^2)) / 2 needs no
  // division, the larger c_f^2 = X / rho is chosen by cross-multiplication,
  // and only its side takes a reciprocal and a root
  auto rho_cf2 = [&](T p, T bb, T bt) {
    const T gp = gamma * p;
    const T dd = gp - bb;
    return T(0.5) * (gp + bb + tsqrt<T>(dd * dd + T(4) * gp * bt));
  };
  const T XL = rho_cf2(wl[4], bbL, btL), XR = rho_cf2(wr[4], bbR, btR);
  const bool lmax = !nonneg_lt<T>(XL * wr[0], XR * wl[0]);
  const T cmax = tsqrt<T>((lmax ? XL : XR) * trcp<T>(lmax ? wl[0] : wr[0]));
  const T SL = min_s<T>(wl[1], wr[1]) - cmax;
  const T SR = max_s<T>(wl[1], wr[1]) + cmax;

  auto phys = [&](const T* w, T e, T pt, T* F) {
    const T mu = w[0] * w[1];
    F[0] = mu;
    F[1] = mu * w[1] + pt - bn2;
    F[2] = mu * w[2] - bn * w[5];
    F[3] = mu * w[3] - bn * w[6];
    F[4] = (e + pt) * w[1] - bn * (w[1] * bn + w[2] * w[5] + w[3] * w[6]);
    F[5] = w[5] * w[1] - bn * w[2];
    F[6] = w[6] * w[1] - bn * w[3];
  };
  // Supersonic faces take the upwind side's physical flux; the others its
  // star or double-star flux.  One physical flux serves both cases, so a
  // warp mixing them evaluates it once.
  const bool sub = !ge0<T>(SL) && !le0<T>(SR);
  T dL = T(0), dR = T(0), rdL = T(0), rdR = T(0), SM = T(0), pts = T(0);
  if (sub) {
    dL = SL - wl[1];
    dR = SR - wr[1];
    rdL = wl[0] * dL;
    rdR = wr[0] * dR;
    const T iden = trcp<T>(rdR - rdL);
    SM = (rdR * wr[1] - rdL * wl[1] - ptR + ptL) * iden;
    pts = (rdR * ptL - rdL * ptR + rdL * rdR * (wr[1] - wl[1])) * iden;
  }
  // the side whose states the flux comes from (ties to the left)
  const bool left = sub ? ge0<T>(SM) : ge0<T>(SL);
  const T* w = left ? wl : wr;
  const T pt = left ? ptL : ptR;
  const T e = energy(w, left ? bbL : bbR);
  T F[7];
  phys(w, e, pt, F);
  if (!sub) {
#pragma unroll
    for (int q = 0; q < 7; ++q) f[q] = F[q];
    return;
  }

  // single-star states of one side: rho*, v*, w*, By*, Bz* (both sides feed
  // the double-star states)
  struct Star {
    T r, v, w, by, bz, sq, rsq, iSM;
  };
  auto star = [&](const T* ws, T S, T d, T rd) {
    Star st;
    st.iSM = trcp<T>(S - SM);
    st.r = rd * st.iSM;
    const T D = rd * (S - SM) - bn2;
    if (abs_lt<T>(D, Eps<T>::hlld * pts)) {
      st.v = ws[2];
      st.w = ws[3];
      st.by = ws[5];
      st.bz = ws[6];
    } else {
      const T iD = trcp<T>(D);
      const T t = bn * (SM - ws[1]) * iD;
      st.v = ws[2] - ws[5] * t;
      st.w = ws[3] - ws[6] * t;
      const T q = (rd * d - bn2) * iD;
      st.by = ws[5] * q;
      st.bz = ws[6] * q;
    }
    st.rsq = trsqrt<T>(st.r);
    st.sq = st.r * st.rsq;
    return st;
  };
  const Star sL = star(wl, SL, dL, rdL);
  const Star sR = star(wr, SR, dR, rdR);

  const Star& s = left ? sL : sR;
  const T S = left ? SL : SR;
  const T d = left ? dL : dR;
  // star energy E* of that side
  const T vb = w[1] * bn + w[2] * w[5] + w[3] * w[6];
  const T vbs = SM * bn + s.v * s.by + s.w * s.bz;
  const T es = (d * e - pt * w[1] + pts * SM + bn * (vb - vbs)) * s.iSM;

  // double-star (rotational) states
  T SsL = SM, SsR = SM;
  T vss, wss, byss, bzss, ess;
  const bool dbl = !nonneg_lt<T>(T(0.5) * bn2, Eps<T>::hlld * pts);
  if (dbl) {
    const T sg = gt0<T>(bn) ? T(1) : T(-1);
    const T abn = fabs(bn);
    SsL = SM - abn * sL.rsq;
    SsR = SM + abn * sR.rsq;
    const T inv = trcp<T>(sL.sq + sR.sq);
    vss = (sL.sq * sL.v + sR.sq * sR.v + (sR.by - sL.by) * sg) * inv;
    wss = (sL.sq * sL.w + sR.sq * sR.w + (sR.bz - sL.bz) * sg) * inv;
    byss = (sL.sq * sR.by + sR.sq * sL.by + sL.sq * sR.sq * (sR.v - sL.v) * sg) * inv;
    bzss = (sL.sq * sR.bz + sR.sq * sL.bz + sL.sq * sR.sq * (sR.w - sL.w) * sg) * inv;
    const T vbss = SM * bn + vss * byss + wss * bzss;
    // E** = E* -+ sqrt(rho*) (v*.B* - v**.B**) sgn(B_n), - on the left
    if (left)
      ess = es - s.sq * (SM * bn + s.v * s.by + s.w * s.bz - vbss) * sg;
    else
      ess = es + s.sq * (SM * bn + s.v * s.by + s.w * s.bz - vbss) * sg;
  }
  const T U0[7] = {w[0], w[0] * w[1], w[0] * w[2], w[0] * w[3], e, w[5], w[6]};
  const T Us[7] = {s.r, s.r * SM, s.r * s.v, s.r * s.w, es, s.by, s.bz};
  // F* = F + S (U* - U)
  for (int q = 0; q < 7; ++q) f[q] = F[q] + S * (Us[q] - U0[q]);
  const T Ss = left ? SsL : SsR;
  const bool inner = left ? lt0<T>(SsL) : ge0<T>(SsR);
  if (dbl && inner) {
    const T Uss[7] = {s.r, s.r * SM, s.r * vss, s.r * wss, ess, byss, bzss};
    for (int q = 0; q < 7; ++q) f[q] = f[q] + Ss * (Uss[q] - Us[q]);
  }
}

// ------------------------------------------------ characteristic projection --
// Primitive eigen-system (rho, u, v, w, P, B_t1, B_t2) of one cell with its
// cell-centred longitudinal field bn.  Waves ordered u-cf, u-ca, u-cs, u,
// u+cs, u+ca, u+cf.  beta = (1,1)/sqrt2 for B_t = 0; alpha_f = 1, alpha_s = 0
// when cf2 = cs2; S = sgn(bn) with sgn(0) = +1.  The left eigenvectors are the
// closed-form inverse of the right ones (rows scaled by 1/(2 a^2) for the
// magnetosonic waves, 1/2 for the Alfven waves).
template <class T> struct Eig {
  T rho, ir, sr, isr, a, a2, ia2, af, as, cf, cs, Qf, Qs, Af, As, b1, b2, sg;
  T rcf;  // 1/c_f (for the reverse sweep)
};

// Square roots and divisions are folded into five reciprocal square roots
// and one square root: 1/sqrt(rho), 1/a, 1/c_f, 1/|B_t|, and
// q = 1/sqrt(2 s (s + |D|)) with s = c_f^2 - c_s^2, D = a^2 - b^2, giving
// c_s = a c_a / c_f and the alpha pair (s + |D|) q, 2 a |b_t| q.
template <class T> __device__ __forceinline__ void eig_build(T gamma, const T* w, T bn, Eig<T>& E) {
  E.rho = w[0];
  E.isr = trsqrt<T>(w[0]);
  E.sr = w[0] * E.isr;
  E.ir = E.isr * E.isr;
  E.a2 = gamma * w[4] * E.ir;
  const T ra = trsqrt<T>(E.a2);
  E.a = E.a2 * ra;
  E.ia2 = ra * ra;
  const T ca2 = bn * bn * E.ir;
  const T bt2r = w[5] * w[5] + w[6] * w[6];
  const T bt2 = bt2r * E.ir;
  const T b2 = ca2 + bt2;
  const T D = E.a2 - b2;
  const T sd = tsqrt<T>(D * D + T(4) * E.a2 * bt2);
  const T cf2 = T(0.5) * (E.a2 + b2 + sd);
  const T rcf = trsqrt<T>(cf2);
  E.rcf = rcf;
  E.cf = cf2 * rcf;
  E.cs = E.a * fabs(bn) * E.isr * rcf;
  const T ibt = gt0<T>(bt2r) ? trsqrt<T>(bt2r) : T(0);
  const T btn = bt2r * ibt * E.isr;  // |B_t| / sqrt(rho)
  // one formula for both signs of D (only the assignment of the two members
  // to alpha_f and alpha_s depends on it), so neighbouring cells with
  // different signs share one path through the FP64 pipe
  if (is0<T>(sd)) {
    E.af = T(1);
    E.as = T(0);
  } else {
    const bool dpos = ge0<T>(D);
    const T sa = sd + absv<T>(D);
    const T q = trsqrt<T>(T(2) * sd * sa);
    const T big = sa * q, small = T(2) * E.a * btn * q;
    E.af = dpos ? big : small;
    E.as = dpos ? small : big;
  }
  if (is0<T>(bt2r)) {
    E.b1 = T(0.70710678118654752440);
    E.b2 = T(0.70710678118654752440);
  } else {
    E.b1 = w[5] * ibt;
    E.b2 = w[6] * ibt;
  }
  E.sg = ge0<T>(bn) ? T(1) : T(-1);
  const T a = E.a;
  E.Qf = E.cf * E.af * E.sg;
  E.Qs = E.cs * E.as * E.sg;
  E.Af = a * E.af * E.sr;
  E.As = a * E.as * E.sr;
}

// characteristic amplitudes q = L dw
template <class T> __device__ __forceinline__ void eig_left(const Eig<T>& E, const T* dw, T* q) {
  const T n = T(0.5) * E.ia2;
  const T ir = E.ir;
  const T bv = E.b1 * dw[2] + E.b2 * dw[3];
  const T bb = (E.b1 * dw[5] + E.b2 * dw[6]) * E.isr;
  const T sa = E.a;
  const T Xf = E.af * dw[4] * ir + E.as * sa * bb;
  const T Yf = -E.af * E.cf * dw[1] + E.Qs * bv;
  const T Xs = E.as * dw[4] * ir - E.af * sa * bb;
  const T Ys = -E.as * E.cs * dw[1] - E.Qf * bv;
  const T Z = T(0.5) * (-E.b2 * dw[2] + E.b1 * dw[3]);
  const T Zb = T(0.5) * E.sg * (-E.b2 * dw[5] + E.b1 * dw[6]) * E.isr;
  q[0] = n * (Xf + Yf);
  q[1] = Z + Zb;
  q[2] = n * (Xs + Ys);
  q[3] = dw[0] - dw[4] * E.ia2;
  q[4] = n * (Xs - Ys);
  q[5] = Z - Zb;
  q[6] = n * (Xf - Yf);
}

// primitive increments dw = R q
template <class T> __device__ __forceinline__ void eig_right(const Eig<T>& E, const T* q, T* dw) {
  const T fp = q[0] + q[6], fm = q[0] - q[6];
  const T sp = q[2] + q[4], sm = q[2] - q[4];
  const T ap = q[1] + q[5], am = q[1] - q[5];
  const T cfa = E.cf * E.af, csa = E.cs * E.as;
  dw[0] = E.rho * (E.af * fp + E.as * sp) + q[3];
  dw[1] = -cfa * fm - csa * sm;
  dw[2] = E.b1 * (E.Qs * fm - E.Qf * sm) - E.b2 * ap;
  dw[3] = E.b2 * (E.Qs * fm - E.Qf * sm) + E.b1 * ap;
  dw[4] = E.rho * E.a2 * (E.af * fp + E.as * sp);
  const T ms = E.As * fp - E.Af * sp;
  const T ssr = E.sg * E.sr * am;
  dw[5] = E.b1 * ms - E.b2 * ssr;
  dw[6] = E.b2 * ms + E.b1 * ssr;
}

template <class T> __device__ __forceinline__ T sgn0(T x) { return x > T(0) ? T(1) : (x < T(0) ? T(-1) : T(0)); }

// Sign tests and magnitude minima of the limiters.  The generic forms use
// floating-point instructions; for double they run on the bit patterns
// (integer pipes), because the FP64 pipe bounds the FP64 step on this GPU.
// Both give the same result for finite values whose products do not
// underflow.
template <class T> __device__ __forceinline__ bool pos_prod(T a, T b) { return a * b > T(0); }
template <class T> __device__ __forceinline__ bool neg_prod(T a, T b) { return a * b < T(0); }
template <class T> __device__ __forceinline__ T min_abs(T a, T b) { return fmin(fabs(a), fabs(b)); }
// sgn0(s) m for m >= 0
template <class T> __device__ __forceinline__ T with_sign(T s, T m) { return sgn0<T>(s) * m; }
template <class T> __device__ __forceinline__ bool abs_ge_twice(T a, T b) { return fabs(a) >= T(2) * fabs(b); }
template <class T> __device__ __forceinline__ T twice(T x) { return T(2) * x; }
template <> __device__ __forceinline__ df twice<df>(df x) { return df(2.0f * x.hi, 2.0f * x.lo); }

template <> __device__ __forceinline__ bool pos_prod<double>(double a, double b) {
  const long long x = dbits(a), y = dbits(b);
  return ((x ^ y) >= 0) & ((x & kAbsBits) != 0) & ((y & kAbsBits) != 0);
}
template <> __device__ __forceinline__ bool neg_prod<double>(double a, double b) {
  const long long x = dbits(a), y = dbits(b);
  return ((x ^ y) < 0) & ((x & kAbsBits) != 0) & ((y & kAbsBits) != 0);
}
template <> __device__ __forceinline__ double min_abs<double>(double a, double b) {
  const long long x = dbits(a) & kAbsBits, y = dbits(b) & kAbsBits;
  return __longlong_as_double(x < y ? x : y);
}
template <> __device__ __forceinline__ double with_sign<double>(double s, double m) {
  const long long x = dbits(s);
  return (x & kAbsBits) ? __longlong_as_double(dbits(m) | (x & ~kAbsBits)) : 0.0;
}
// |a| >= 2 |b|: the exponent of |b| raised by one (normal b; b = 0 stays 0)
template <> __device__ __forceinline__ bool abs_ge_twice<double>(double a, double b) {
  const long long x = dbits(a) & kAbsBits, y = dbits(b) & kAbsBits;
  return x >= (y ? y + (1LL << 52) : 0LL);
}
template <> __device__ __forceinline__ double twice<double>(double v) {
  const long long x = dbits(v);
  return (x & kAbsBits) ? __longlong_as_double(x + (1LL << 52)) : v;
}

// ------------------------------------------------------- PLMC (Sec. 2.2.6) --
// wm, w0, wp: primitive 7-vectors of cells i-1, i, i+1; bn: cell-centred
// longitudinal field of cell i.  Outputs W_{L,i+1/2} and W_{R,i-1/2}.
// van Leer differences dG = 2 dL dR / (dL + dR) where dL dR > 0, else 0
// (reading D-5), for the 7 fields of one cell
template <class T> __device__ __forceinline__ void van_leer7(const T* dL, const T* dR, T* dG) {
#pragma unroll
  for (int q = 0; q < 7; ++q)
    dG[q] = pos_prod<T>(dL[q], dR[q]) ? T(2) * (dL[q] * dR[q]) * trcp<T>(dL[q] + dR[q]) : T(0);
}
// Double: the seven reciprocals from one (Montgomery's simultaneous
// inversion: prefix products, one reciprocal, back-substitution), when every
// denominator lies in [2^-140, 2^140] so that no partial product leaves the
// normal range; otherwise one reciprocal each.  The FP64 pipe bounds the
// FP64 step and a reciprocal costs about 7 of its multiplies.
static __device__ __noinline__ void rcp7_call(const double* s, double* inv) {
#pragma unroll
  for (int q = 0; q < 7; ++q) inv[q] = trcp<double>(s[q]);
}
template <> __device__ __forceinline__ void van_leer7<double>(const double* dL, const double* dR, double* dG) {
  double s[7], p[7], inv[7];
  bool act[7];
  bool ok = true;
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    act[q] = pos_prod<double>(dL[q], dR[q]);
    s[q] = act[q] ? dL[q] + dR[q] : 1.0;
    const long long e = (dbits(s[q]) >> 52) & 0x7ff;
    ok &= (e >= 1023 - 140) & (e <= 1023 + 140);
  }
  p[0] = s[0];
#pragma unroll
  for (int q = 1; q < 7; ++q) p[q] = p[q - 1] * s[q];
  double r = trcp<double>(p[6]);
#pragma unroll
  for (int q = 6; q > 0; --q) {
    inv[q] = r * p[q - 1];
    r = r * s[q];
  }
  inv[0] = r;
  // the rare fallback is a call made only in warps where some lane needs it
  if (__any_sync(__activemask(), !ok)) {
    if (!ok) rcp7_call(s, inv);
  }
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    // (a product that underflows gives 0, also where 1/s would overflow)
    const double pr = dL[q] * dR[q];
    dG[q] = (act[q] && (dbits(pr) & kAbsBits) != 0) ? twice<double>(pr) * inv[q] : 0.0;
  }
}

template <class T>
__device__ __forceinline__ void plmc(T gamma, const T* wm, const T* w0, const T* wp, T bn, T* wl, T* wr) {
  T dL[7], dR[7], dG[7];
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    dL[q] = w0[q] - wm[q];
    dR[q] = wp[q] - w0[q];
  }
  van_leer7<T>(dL, dR, dG);
  Eig<T> E;
  eig_build<T>(gamma, w0, bn, E);
  T aL[7], aR[7], aC[7], aG[7], am[7], dW[7];
  eig_left<T>(E, dL, aL);
  eig_left<T>(E, dR, aR);
  eig_left<T>(E, dG, aG);
  // the centred difference (W_{i+1} - W_{i-1})/2 projected: L is linear, so
  // its amplitudes are the mean of the left and right ones
#pragma unroll
  for (int q = 0; q < 7; ++q) aC[q] = T(0.5) * (aL[q] + aR[q]);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    if (pos_prod<T>(aL[q], aR[q])) {
      const T m = min_abs<T>(min_abs<T>(twice<T>(aL[q]), twice<T>(aR[q])), min_abs<T>(aC[q], aG[q]));
      am[q] = with_sign<T>(aC[q], m);
    } else {
      am[q] = T(0);
    }
  }
  eig_right<T>(E, am, dW);
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    wl[q] = w0[q] + T(0.5) * dW[q];
    wr[q] = w0[q] - T(0.5) * dW[q];
  }
}

// PLM with the limiter applied to the primitive differences themselves (the
// variant named at the end of Sec. 2.2.6): the same slopes and limiter as
// plmc, without the characteristic projection.
template <class T>
__device__ __forceinline__ void plm_prim(const T* wm, const T* w0, const T* wp, T* wl, T* wr) {
#pragma unroll
  for (int q = 0; q < 7; ++q) {
    const T dL = w0[q] - wm[q], dR = wp[q] - w0[q], dC = T(0.5) * (wp[q] - wm[q]);
    const T pr = dL * dR;
    T dm = T(0);
    if (pr > T(0)) {
      const T dG = T(2) * pr * trcp<T>(dL + dR);
      dm = sgn0<T>(dC) * fmin(fmin(T(2) * fabs(dL), T(2) * fabs(dR)), fmin(fabs(dC), fabs(dG)));
    }
    wl[q] = w0[q] + T(0.5) * dm;
    wr[q] = w0[q] - T(0.5) * dm;
  }
}

// ------------------------------------------------------- PPMC (Sec. 2.2.6) --
// Fourth-order interface values, Colella & Sekora (2008) interface limiter,
// McCorquodale & Colella (2011) cell limiter (C = 1.25), in characteristic
// deviations q_m - q_0 = L (W_m - W_0) of cell i.
// sgn(x) min(|x|, C|y|, C|z|) when x, y, z share a strict sign, else 0 (C = 1.25)
// (C min(|y|, |z|) is min(C|y|, C|z|) exactly: a rounded product is monotone)
template <class T> __device__ __forceinline__ T d2lim3(T x, T y, T z) {
  if (pos_prod<T>(x, y) && pos_prod<T>(x, z))
    return with_sign<T>(x, min_abs<T>(x, T(1.25) * min_abs<T>(y, z)));
  return T(0);
}
template <class T> __device__ __forceinline__ T d2lim4(T x, T y, T z, T t) {
  if (pos_prod<T>(x, y) && pos_prod<T>(x, z) && pos_prod<T>(x, t))
    return with_sign<T>(x, min_abs<T>(x, T(1.25) * min_abs<T>(y, min_abs<T>(z, t))));
  return T(0);
}

// a / b for |a| <= |b|, b != 0
template <class T> __device__ __forceinline__ T ratio_le1(T a, T b) { return a / b; }
static __device__ __noinline__ double div_call(double a, double b) { return a / b; }
template <> __device__ __forceinline__ double ratio_le1<double>(double a, double b) {
  // biased exponent >= 64: 1/b is finite and normal.  The division for
  // smaller b is a call made only in warps where some lane needs it (inlined,
  // the compiler evaluates it in every warp, on the FP64 pipe)
  const bool tiny = ((dbits(b) >> 52) & 0x7ff) < 64;
  double r = a * trcp<double>(b);
  if (__any_sync(__activemask(), tiny)) {
    if (tiny) r = div_call(a, b);
  }
  return r;
}

// q[0..4] = characteristic deviations of cells i-2..i+2 from cell i (q[2] = 0);
// returns the limited deviations of the two interface values.  Written for
// the deviation form: the centre's zero is not added, subtracted or
// multiplied, and sign flips and doublings are exact bit operations, so
// only the arithmetic the limiter needs reaches the FP64 pipe.  Same values
// as the formulas with q[2] kept, up to the sign of zero results.
template <class T> __device__ __forceinline__ T neg(T x) { return -x; }
template <> __device__ __forceinline__ double neg<double>(double x) { return __longlong_as_double(dbits(x) ^ kNegZero); }
template <class T> __device__ __forceinline__ void ppm_one(const T* q, T& qm, T& qp) {
  const T c7 = from_d<T>(7.0 / 12.0), c1 = from_d<T>(1.0 / 12.0), c6 = from_d<T>(1.0 / 6.0);
  const T a = q[0], b = q[1], d = q[3], e = q[4];  // cells i-2, i-1, i+1, i+2
  qm = c7 * b - c1 * (a + d);
  qp = c7 * d - c1 * (b + e);
  const T d2m1 = a - T(2) * b;
  const T d20 = b + d;
  const T d2p1 = e - T(2) * d;
  // interface limiter where the value leaves the range of its two cells.
  // Both interfaces share one body, fed the operands of the lower interface
  // where it needs limiting, else of the upper: a warp whose lanes limit
  // different interfaces runs it once; a second pass runs only where a lane
  // limits both.
  const bool lm = pos_prod<T>(qm - b, qm), lp = neg_prod<T>(qp, d - qp);
  if (lm || lp) {
    const T x = lm ? b : d, v = lm ? qm : qp, y = lm ? d2m1 : d20, z = lm ? d20 : d2p1;
    const T lim = T(0.5) * x - d2lim3<T>(T(3) * (x - T(2) * v), y, z) * c6;
    if (lm) qm = lim;
    else qp = lim;
    if (lm && lp) qp = T(0.5) * d - d2lim3<T>(T(3) * (d - T(2) * qp), d20, d2p1) * c6;
  }
  // cell limiter: at an extremum both deviations scale by the curvature
  // ratio, elsewhere an overshoot is clipped to twice the other deviation
  if (!neg_prod<T>(qm, qp) || !neg_prod<T>(b, d)) {
    const T d2f = T(6) * (qm + qp);
    T r = T(0);
    // (|d2lim4 / d2f| <= 1: a reciprocal where d2f is far from the
    // underflow range, else the division)
    if (!is0<T>(d2f)) r = ratio_le1<T>(d2lim4<T>(d2f, d2m1, d20, d2p1), d2f);
    qm = r * qm;
    qp = r * qp;
  } else {
    const T m0 = qm;
    if (abs_ge_twice<T>(qm, qp)) qm = neg<T>(twice<T>(qp));
    if (abs_ge_twice<T>(qp, m0)) qp = neg<T>(twice<T>(m0));
  }
}

template <class T>
__device__ __forceinline__ void ppmc(T gamma, const T (*w)[7], T bn, T* wl, T* wr) {
  Eig<T> E;
  eig_build<T>(gamma, w[2], bn, E);
  T qs[5][7];
#pragma unroll
  for (int m = 0; m < 5; ++m) {
    if (m == 2) {
#pragma unroll
      for (int c = 0; c < 7; ++c) qs[2][c] = T(0);
      continue;
    }
    T d[7];
#pragma unroll
    for (int c = 0; c < 7; ++c) d[c] = w[m][c] - w[2][c];
    eig_left<T>(E, d, qs[m]);
  }
  T dm[7], dp[7];
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    const T col[5] = {qs[0][c], qs[1][c], T(0), qs[3][c], qs[4][c]};
    T qm, qp;
    ppm_one<T>(col, qm, qp);
    dm[c] = qm;
    dp[c] = qp;
  }
  T Wm[7], Wp[7];
  eig_right<T>(E, dm, Wm);
  eig_right<T>(E, dp, Wp);
#pragma unroll
  for (int c = 0; c < 7; ++c) {
    wl[c] = w[2][c] + Wp[c];
    wr[c] = w[2][c] + Wm[c];
  }
}

}  // namespace mhd
