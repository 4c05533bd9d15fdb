// mhd_oracle.cpp -- plain, slow FP64 CPU oracle of the VL+CT ideal-MHD step.
//
// TEST INFRASTRUCTURE ONLY.  This file is the reference that the CUDA path is
// checked against.  Only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline leg may load it.  It shares no code, header, table or helper
// with the CUDA library; neither includes or links the other.
//
// Method: Caddy & Schneider, "Cholla-MHD" (arXiv:2402.05240), Sec. 2.2 (VL+CT
// integrator, Steps 1-10), Sec. 2.1 (equations and fluxes), Table "emf"
// (flux -> face electric field), with the HLLD solver of Miyoshi & Kusano
// (2005), the primitive eigenvectors of Stone et al. (2008, App. A) and the
// PPM limiters of Colella & Sekora (2008) / McCorquodale & Colella (2011) in
// characteristic variables (Felker & Stone 2018), all written from the
// published definitions.  Readings of ambiguous passages are labelled D-n.
//
// Everything is written as plain loops over all cells with periodic (modular)
// indices; no blocking, fusion or reordering.  Scalar code is templated on the
// number type so that the same source runs in double and in a forward-mode
// dual number (value + one directional derivative) for Jacobian-vector
// product references; branch decisions always use the value part.
//
// Layout: U[8][nz][ny][nx] double, fields rho, mx, my, mz, E, Bx, By, Bz;
// Bx[k][j][i] is the face value at x_{i+1/2} (Sec. 2.2, staggered grid).
//
// parity pinned: see tests/test_oracle_*.py for the pins of each function.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ---------------------------------------------------------------- scalars --
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double x) : v(x), d(0) {}
  Dual(double x, double dx) : v(x), d(dx) {}
};
inline Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
inline Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
inline Dual operator-(Dual a) { return {-a.v, -a.d}; }
inline Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return {q, (a.d - q * b.d) / b.v};
}
inline Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
inline Dual operator+(double a, Dual b) { return {a + b.v, b.d}; }
inline Dual operator-(Dual a, double b) { return {a.v - b, a.d}; }
inline Dual operator-(double a, Dual b) { return {a - b.v, -b.d}; }
inline Dual operator*(Dual a, double b) { return {a.v * b, a.d * b}; }
inline Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
inline Dual operator/(Dual a, double b) { return {a.v / b, a.d / b}; }
inline Dual operator/(double a, Dual b) {
  double q = a / b.v;
  return {q, -q * b.d / b.v};
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }

inline double val(double x) { return x; }
inline double val(const Dual& x) { return x.v; }
inline double S_sqrt(double x) { return std::sqrt(x); }
inline Dual S_sqrt(Dual x) {
  double s = std::sqrt(x.v);
  return {s, s > 0 ? 0.5 * x.d / s : 0.0};
}
template <class S> inline S S_abs(const S& x) { return val(x) < 0 ? S(-x) : x; }
template <class S> inline S S_max(const S& a, const S& b) { return val(a) >= val(b) ? a : b; }
template <class S> inline S S_min(const S& a, const S& b) { return val(a) <= val(b) ? a : b; }
// sign with sgn(0) = 0
template <class S> inline double sgn0(const S& x) { return val(x) > 0 ? 1.0 : (val(x) < 0 ? -1.0 : 0.0); }

// ------------------------------------------------------------------- grid --
struct Params {  // mirrored by ctypes in oracle/__init__.py
  int n[3];
  double d[3];
  double gamma;
  double rho_floor, p_floor;
  int recon;  // 0 PCM, 1 PLMC, 2 PPMC
};

inline int wrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

struct Grid {
  int n[3];
  long N;
  explicit Grid(const Params& p) {
    for (int a = 0; a < 3; ++a) n[a] = p.n[a];
    N = (long)n[0] * n[1] * n[2];
  }
  long at(int i, int j, int k) const {
    return ((long)wrap(k, n[2]) * n[1] + wrap(j, n[1])) * n[0] + wrap(i, n[0]);
  }
  long at(const int* p) const { return at(p[0], p[1], p[2]); }
  // cell index of p + s * e_a (+ t * e_b)
  long shift(const int* p, int a, int s) const {
    int q[3] = {p[0], p[1], p[2]};
    q[a] += s;
    return at(q);
  }
  long shift2(const int* p, int a, int s, int b, int t) const {
    int q[3] = {p[0], p[1], p[2]};
    q[a] += s;
    q[b] += t;
    return at(q);
  }
  void coords(long c, int* p) const {
    p[0] = (int)(c % n[0]);
    p[1] = (int)((c / n[0]) % n[1]);
    p[2] = (int)(c / ((long)n[0] * n[1]));
  }
};

// ------------------------------------------------------ O1. primitives ----
// Cell-centred B is the mean of the two faces (Sec. 2.2.1); v = m/rho;
// P = (gamma-1)(E - |m|^2/(2 rho) - |B|^2/2) (Sec. 2.1, ideal gas).
// Floors (D-12): rho and P are raised to rho_floor / p_floor before use.
template <class S> struct Prim {
  S rho, v[3], p, b[3];
};

template <class S>
Prim<S> primitive(const Params& P, const Grid& g, const S* U, const int* p) {
  const long N = g.N;
  const long c = g.at(p);
  Prim<S> w;
  for (int a = 0; a < 3; ++a) w.b[a] = 0.5 * (U[(5 + a) * N + g.shift(p, a, -1)] + U[(5 + a) * N + c]);
  w.rho = S_max(U[c], S(P.rho_floor));
  S m[3] = {U[N + c], U[2 * N + c], U[3 * N + c]};
  for (int a = 0; a < 3; ++a) w.v[a] = m[a] / w.rho;
  S ke = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / w.rho;
  S me = 0.5 * (w.b[0] * w.b[0] + w.b[1] * w.b[1] + w.b[2] * w.b[2]);
  w.p = (P.gamma - 1.0) * (U[4 * N + c] - ke - me);
  w.p = S_max(w.p, S(P.p_floor));
  return w;
}

// 7-vector in the solver frame of axis a: (rho, v_n, v_t1, v_t2, P, B_t1, B_t2)
// with (n, t1, t2) = (a, a+1, a+2) cyclically (Table "emf" note).
template <class S> void directional(const Prim<S>& w, int a, S* out, S* bn_cc) {
  int b = (a + 1) % 3, c = (a + 2) % 3;
  out[0] = w.rho;
  out[1] = w.v[a];
  out[2] = w.v[b];
  out[3] = w.v[c];
  out[4] = w.p;
  out[5] = w.b[b];
  out[6] = w.b[c];
  *bn_cc = w.b[a];
}

// Fast magnetosonic speed with longitudinal field bl (Sec. 2.2.1 c_f formula,
// D-8: per direction).  The discriminant (gamma P + B^2)^2 - 4 gamma P B_l^2
// (divided by rho^2) is written as the equal sum of non-negative terms
// (a2 - b2)^2 + 4 a2 bt2, a2 = gamma P/rho, b2 = |B|^2/rho, bt2 = B_t^2/rho.
template <class S> S fast_speed(double gamma, const S& rho, const S& p, const S& bl, const S& bt1, const S& bt2) {
  S a2 = gamma * p / rho;
  S t2 = (bt1 * bt1 + bt2 * bt2) / rho;
  S b2 = bl * bl / rho + t2;
  S disc = (a2 - b2) * (a2 - b2) + 4.0 * a2 * t2;
  return S_sqrt(0.5 * (a2 + b2 + S_sqrt(disc)));
}

// ----------------------------------------------------------------- O4. HLLD --
// Miyoshi & Kusano (2005), solver frame, state (rho, u, v, w, P, By, Bz), Bx = bn.
// Degeneracy threshold relative to p_T* (D-9): 1e-8.
constexpr double kHlldEps = 1e-8;

template <class S> struct Cons7 { S q[7]; };

template <class S> struct HlldDetail {
  S SL, SsL, SM, SsR, SR;
  S UL[7], UsL[7], UssL[7], UssR[7], UsR[7], UR[7];
  S FL[7], FR[7];
  bool star;  // star states were formed (SL < 0 < SR)
};

template <class S>
void physical(double gamma, const S* w, const S& bn, S* U, S* F, S* pt_out) {
  const S &rho = w[0], &u = w[1], &v = w[2], &ww = w[3], &p = w[4], &by = w[5], &bz = w[6];
  S b2 = bn * bn + by * by + bz * bz;
  S e = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + ww * ww) + 0.5 * b2;
  S pt = p + 0.5 * b2;
  U[0] = rho;
  U[1] = rho * u;
  U[2] = rho * v;
  U[3] = rho * ww;
  U[4] = e;
  U[5] = by;
  U[6] = bz;
  // F_x of Sec. 2.1 in the solver frame
  F[0] = rho * u;
  F[1] = rho * u * u + pt - bn * bn;
  F[2] = rho * u * v - bn * by;
  F[3] = rho * u * ww - bn * bz;
  F[4] = (e + pt) * u - bn * (u * bn + v * by + ww * bz);
  F[5] = by * u - bn * v;
  F[6] = bz * u - bn * ww;
  *pt_out = pt;
}

template <class S>
void hlld(double gamma, const S* wl, const S* wr, const S& bn, S* flux, HlldDetail<S>* det = nullptr) {
  S UL[7], UR[7], FL[7], FR[7], ptL, ptR;
  physical(gamma, wl, bn, UL, FL, &ptL);
  physical(gamma, wr, bn, UR, FR, &ptR);
  S cfL = fast_speed(gamma, wl[0], wl[4], bn, wl[5], wl[6]);
  S cfR = fast_speed(gamma, wr[0], wr[4], bn, wr[5], wr[6]);
  S cmax = S_max(cfL, cfR);
  S SL = S_min(wl[1], wr[1]) - cmax;
  S SR = S_max(wl[1], wr[1]) + cmax;
  if (det) {
    det->SL = SL;
    det->SR = SR;
    det->star = false;
    for (int q = 0; q < 7; ++q) {
      det->UL[q] = UL[q];
      det->UR[q] = UR[q];
      det->FL[q] = FL[q];
      det->FR[q] = FR[q];
    }
  }
  if (val(SL) >= 0) {
    for (int q = 0; q < 7; ++q) flux[q] = FL[q];
    return;
  }
  if (val(SR) <= 0) {
    for (int q = 0; q < 7; ++q) flux[q] = FR[q];
    return;
  }
  const S &rL = wl[0], &uL = wl[1], &rR = wr[0], &uR = wr[1];
  S dL = SL - uL, dR = SR - uR;
  S den = dR * rR - dL * rL;
  S SM = (dR * rR * uR - dL * rL * uL - ptR + ptL) / den;            // MK05 eq. (38)
  S pts = (dR * rR * ptL - dL * rL * ptR + rL * rR * dR * dL * (uR - uL)) / den;  // eq. (41)

  // single-star states, eqs. (43)-(48)
  S Us[2][7], Uss[2][7], sqr[2], vs[2], ws[2], bys[2], bzs[2], es[2];
  const S* wv[2] = {wl, wr};
  const S* Uv[2] = {UL, UR};
  S Sv[2] = {SL, SR};
  S dv[2] = {dL, dR};
  S ptv[2] = {ptL, ptR};
  for (int s = 0; s < 2; ++s) {
    const S* w = wv[s];
    const S &rho = w[0], &u = w[1], &v = w[2], &ww = w[3], &by = w[5], &bz = w[6];
    S rs = rho * dv[s] / (Sv[s] - SM);
    S D = rho * dv[s] * (Sv[s] - SM) - bn * bn;
    if (val(S_abs(D)) < kHlldEps * val(pts)) {
      vs[s] = v;
      ws[s] = ww;
      bys[s] = by;
      bzs[s] = bz;
    } else {
      S t = bn * (SM - u) / D;
      vs[s] = v - by * t;
      ws[s] = ww - bz * t;
      S f = (rho * dv[s] * dv[s] - bn * bn) / D;
      bys[s] = by * f;
      bzs[s] = bz * f;
    }
    S vb = u * bn + v * by + ww * bz;
    S vbs = SM * bn + vs[s] * bys[s] + ws[s] * bzs[s];
    es[s] = (dv[s] * Uv[s][4] - ptv[s] * u + pts * SM + bn * (vb - vbs)) / (Sv[s] - SM);
    Us[s][0] = rs;
    Us[s][1] = rs * SM;
    Us[s][2] = rs * vs[s];
    Us[s][3] = rs * ws[s];
    Us[s][4] = es[s];
    Us[s][5] = bys[s];
    Us[s][6] = bzs[s];
    sqr[s] = S_sqrt(rs);
  }
  // double-star states, eqs. (49)-(63)
  S SsL = SM, SsR = SM;
  if (val(0.5 * bn * bn) < kHlldEps * val(pts)) {
    for (int s = 0; s < 2; ++s)
      for (int q = 0; q < 7; ++q) Uss[s][q] = Us[s][q];
  } else {
    double sg = val(bn) > 0 ? 1.0 : -1.0;
    S abn = S_abs(bn);
    SsL = SM - abn / sqr[0];
    SsR = SM + abn / sqr[1];
    S inv = 1.0 / (sqr[0] + sqr[1]);
    S vss = (sqr[0] * vs[0] + sqr[1] * vs[1] + (bys[1] - bys[0]) * sg) * inv;
    S wss = (sqr[0] * ws[0] + sqr[1] * ws[1] + (bzs[1] - bzs[0]) * sg) * inv;
    S byss = (sqr[0] * bys[1] + sqr[1] * bys[0] + sqr[0] * sqr[1] * (vs[1] - vs[0]) * sg) * inv;
    S bzss = (sqr[0] * bzs[1] + sqr[1] * bzs[0] + sqr[0] * sqr[1] * (ws[1] - ws[0]) * sg) * inv;
    S vbss = SM * bn + vss * byss + wss * bzss;
    for (int s = 0; s < 2; ++s) {
      S vbs = SM * bn + vs[s] * bys[s] + ws[s] * bzs[s];
      double side = s == 0 ? -1.0 : 1.0;
      S ess = es[s] + side * sqr[s] * (vbs - vbss) * sg;
      S rs = Us[s][0];
      Uss[s][0] = rs;
      Uss[s][1] = rs * SM;
      Uss[s][2] = rs * vss;
      Uss[s][3] = rs * wss;
      Uss[s][4] = ess;
      Uss[s][5] = byss;
      Uss[s][6] = bzss;
    }
  }
  if (det) {
    det->star = true;
    det->SsL = SsL;
    det->SM = SM;
    det->SsR = SsR;
    for (int q = 0; q < 7; ++q) {
      det->UsL[q] = Us[0][q];
      det->UssL[q] = Uss[0][q];
      det->UssR[q] = Uss[1][q];
      det->UsR[q] = Us[1][q];
    }
  }
  // flux selection, ties to the left branch (O4)
  for (int q = 0; q < 7; ++q) {
    S FsL = FL[q] + SL * (Us[0][q] - UL[q]);
    S FsR = FR[q] + SR * (Us[1][q] - UR[q]);
    if (val(SsL) >= 0)
      flux[q] = FsL;
    else if (val(SM) >= 0)
      flux[q] = FsL + SsL * (Uss[0][q] - Us[0][q]);
    else if (val(SsR) >= 0)
      flux[q] = FsR + SsR * (Uss[1][q] - Us[1][q]);
    else
      flux[q] = FsR;
  }
}

// ------------------------------------------------------- O9. eigensystem --
// Right eigenvectors of the primitive system (rho, u, v, w, P, By, Bz) in the
// normalisation of Stone et al. (2008, App. A); columns ordered by
// lambda = u-cf, u-ca, u-cs, u, u+cs, u+ca, u+cf.  D-10 conventions:
// beta = (1,1)/sqrt2 when B_t = 0; alpha_f = 1, alpha_s = 0 when cf2 = cs2;
// S = sgn(B_n) with sgn(0) = +1.  L = R^-1 by Gaussian elimination, with the
// elimination's round-off in exactly-zero entries removed.
template <class S> struct Eigen {
  S lam[7];
  S R[7][7];  // R[row][col]
  S L[7][7];
};

template <class S> void invert7(S A[7][7], S X[7][7]) {
  S M[7][14];
  for (int i = 0; i < 7; ++i)
    for (int j = 0; j < 7; ++j) {
      M[i][j] = A[i][j];
      M[i][7 + j] = S(i == j ? 1.0 : 0.0);
    }
  for (int col = 0; col < 7; ++col) {
    int piv = col;
    for (int r = col + 1; r < 7; ++r)
      if (std::fabs(val(M[r][col])) > std::fabs(val(M[piv][col]))) piv = r;
    if (piv != col)
      for (int j = 0; j < 14; ++j) std::swap(M[piv][j], M[col][j]);
    S inv = 1.0 / M[col][col];
    for (int j = 0; j < 14; ++j) M[col][j] = M[col][j] * inv;
    for (int r = 0; r < 7; ++r) {
      if (r == col) continue;
      S f = M[r][col];
      for (int j = 0; j < 14; ++j) M[r][j] = M[r][j] - f * M[col][j];
    }
  }
  for (int i = 0; i < 7; ++i)
    for (int j = 0; j < 7; ++j) X[i][j] = M[i][7 + j];
}


template <class S> void eigensystem(double gamma, const S* w, const S& bn, Eigen<S>& E) {
  const S &rho = w[0], &u = w[1], &p = w[4], &by = w[5], &bz = w[6];
  S a2 = gamma * p / rho;
  S ca2 = bn * bn / rho;
  S bt2 = (by * by + bz * bz) / rho;
  S b2 = ca2 + bt2;
  S D = a2 - b2;
  S sd = S_sqrt(D * D + 4.0 * a2 * bt2);  // cf2 - cs2
  S cf2 = 0.5 * (a2 + b2 + sd);
  S cs2 = a2 * ca2 / cf2;
  S cf = S_sqrt(cf2), cs = S_sqrt(cs2), a = S_sqrt(a2), ca = S_sqrt(ca2);
  S bt = S_sqrt(by * by + bz * bz);
  S b1, b2n;
  if (val(bt) == 0.0) {
    b1 = S(1.0 / std::sqrt(2.0));
    b2n = S(1.0 / std::sqrt(2.0));
  } else {
    b1 = by / bt;
    b2n = bz / bt;
  }
  // alpha_f^2 = (a2 - cs2)/(cf2 - cs2) = (sd + D)/(2 sd), alpha_s^2 = (sd - D)/(2 sd);
  // the member that cancels is rewritten as 2 a2 bt2 / (sd (sd + |D|)).
  S af, as;
  if (val(sd) == 0.0) {
    af = S(1.0);
    as = S(0.0);
  } else if (val(D) >= 0) {
    af = S_sqrt((sd + D) / (2.0 * sd));
    as = S_sqrt(2.0 * a2 * bt2 / (sd * (sd + D)));
  } else {
    af = S_sqrt(2.0 * a2 * bt2 / (sd * (sd - D)));
    as = S_sqrt((sd - D) / (2.0 * sd));
  }
  double sg = val(bn) >= 0 ? 1.0 : -1.0;
  S sr = S_sqrt(rho);
  S Cf = cf * af, Cs = cs * as, Qf = Cf * sg, Qs = Cs * sg, Af = a * af * sr, As = a * as * sr;
  S lam[7] = {u - cf, u - ca, u - cs, u, u + cs, u + ca, u + cf};
  for (int i = 0; i < 7; ++i) {
    E.lam[i] = lam[i];
    for (int j = 0; j < 7; ++j) E.R[i][j] = S(0.0);
  }
  // fast waves (columns 0 and 6)
  for (int s = 0; s < 2; ++s) {
    int col = s == 0 ? 0 : 6;
    double pm = s == 0 ? 1.0 : -1.0;  // upper sign for u - cf
    E.R[0][col] = rho * af;
    E.R[1][col] = -pm * Cf;
    E.R[2][col] = pm * Qs * b1;
    E.R[3][col] = pm * Qs * b2n;
    E.R[4][col] = rho * a2 * af;
    E.R[5][col] = As * b1;
    E.R[6][col] = As * b2n;
  }
  // Alfven waves (columns 1 and 5)
  for (int s = 0; s < 2; ++s) {
    int col = s == 0 ? 1 : 5;
    double pm = s == 0 ? 1.0 : -1.0;
    E.R[2][col] = -b2n;
    E.R[3][col] = b1;
    E.R[5][col] = -pm * sg * sr * b2n;
    E.R[6][col] = pm * sg * sr * b1;
  }
  // slow waves (columns 2 and 4)
  for (int s = 0; s < 2; ++s) {
    int col = s == 0 ? 2 : 4;
    double pm = s == 0 ? 1.0 : -1.0;
    E.R[0][col] = rho * as;
    E.R[1][col] = -pm * Cs;
    E.R[2][col] = -pm * Qf * b1;
    E.R[3][col] = -pm * Qf * b2n;
    E.R[4][col] = rho * a2 * as;
    E.R[5][col] = -Af * b1;
    E.R[6][col] = -Af * b2n;
  }
  // entropy wave (column 3)
  E.R[0][3] = S(1.0);
  invert7(E.R, E.L);
  // Entries of R^-1 that are exactly zero (the v_n entries of the slow and
  // entropy rows when B_n = 0, the beta_2 entries when B_t2 = 0, ...) come out
  // of the elimination as O(eps) noise.  The limiters branch on the signs of
  // L dW, so such noise would decide ties that are exact in exact arithmetic:
  // entries below 32 eps of their row's largest entry are set to zero.
  for (int i = 0; i < 7; ++i) {
    double m = 0.0;
    for (int j = 0; j < 7; ++j) m = std::max(m, std::fabs(val(E.L[i][j])));
    for (int j = 0; j < 7; ++j)
      if (std::fabs(val(E.L[i][j])) < 32.0 * 2.220446049250313e-16 * m) E.L[i][j] = S(0.0);
  }
}

template <class S> void matvec7(const S M[7][7], const S* x, S* y) {
  for (int i = 0; i < 7; ++i) {
    S acc = 0.0;
    for (int j = 0; j < 7; ++j) acc += M[i][j] * x[j];
    y[i] = acc;
  }
}

// Directional primitive 7-vector of cell p + s e_a and its cell-centred B_a.
template <class S>
void dir_state(const Params& P, const Grid& g, const S* U, const int* p, int a, int s, S* w, S* bn) {
  int q[3] = {p[0], p[1], p[2]};
  q[a] += s;
  Prim<S> pr = primitive(P, g, U, q);
  directional(pr, a, w, bn);
}

template <class S> void floor_state(const Params& P, S* w) {
  w[0] = S_max(w[0], S(P.rho_floor));
  w[4] = S_max(w[4], S(P.p_floor));
}

// --------------------------------------------------------------- O8. PLMC --
// Sec. 2.2.6 steps 1-6: left/right/centred/van Leer differences of the
// primitives (D-5: van Leer of the differences), projection with the left
// eigenvectors of cell i, the limiter of Eq. "limiter", back-projection and
// W_{L,i+1/2} = W_i + dW/2, W_{R,i-1/2} = W_i - dW/2.  No characteristic
// tracing, no extra clamp (D-13).  prim_limit=true limits the primitive
// differences directly (Sec. 2.2.6, last sentence: skip steps 3 and 5).
template <class S>
void plmc(const Params& P, const Grid& g, const S* U, const int* p, int a, S* wl_out, S* wr_out,
          bool prim_limit = false) {
  S wm[7], w0[7], wp[7], bn, tmp;
  dir_state(P, g, U, p, a, -1, wm, &tmp);
  dir_state(P, g, U, p, a, 0, w0, &bn);
  dir_state(P, g, U, p, a, +1, wp, &tmp);
  S dL[7], dR[7], dC[7], dG[7];
  for (int q = 0; q < 7; ++q) {
    dL[q] = w0[q] - wm[q];
    dR[q] = wp[q] - w0[q];
    dC[q] = 0.5 * (wp[q] - wm[q]);
    dG[q] = val(dL[q] * dR[q]) > 0 ? S(2.0 * dL[q] * dR[q] / (dL[q] + dR[q])) : S(0.0);
  }
  S aL[7], aR[7], aC[7], aG[7], am[7], dW[7];
  Eigen<S> E;
  if (!prim_limit) {
    eigensystem(P.gamma, w0, bn, E);
    matvec7(E.L, dL, aL);
    matvec7(E.L, dR, aR);
    matvec7(E.L, dC, aC);
    matvec7(E.L, dG, aG);
  } else {
    for (int q = 0; q < 7; ++q) {
      aL[q] = dL[q];
      aR[q] = dR[q];
      aC[q] = dC[q];
      aG[q] = dG[q];
    }
  }
  for (int q = 0; q < 7; ++q) {
    if (val(aL[q] * aR[q]) > 0) {
      S m = S_min(S_min(2.0 * S_abs(aL[q]), 2.0 * S_abs(aR[q])), S_min(S_abs(aC[q]), S_abs(aG[q])));
      am[q] = sgn0(aC[q]) * m;
    } else {
      am[q] = S(0.0);
    }
  }
  if (!prim_limit)
    matvec7(E.R, am, dW);
  else
    for (int q = 0; q < 7; ++q) dW[q] = am[q];
  for (int q = 0; q < 7; ++q) {
    wl_out[q] = w0[q] + 0.5 * dW[q];
    wr_out[q] = w0[q] - 0.5 * dW[q];
  }
  floor_state(P, wl_out);
  floor_state(P, wr_out);
}

// --------------------------------------------------------------- O10. PPMC --
// Felker & Stone (2018) PPM in the characteristic variables of cell i:
// (1) project W_{i-2..i+2} - W_i with L(W_i); (2) fourth-order interface values
// q_{i-1/2} = 7/12 (q_{i-1}+q_i) - 1/12 (q_{i-2}+q_{i+1}); (3) Colella & Sekora
// (2008) interface limiter with C = 1.25; (4) McCorquodale & Colella (2011)
// cell limiter; (5) back-projection of the deviations with R(W_i).  D-11.
constexpr double kPpmC = 1.25;

template <class S> S d2lim3(const S& x, const S& y, const S& z) {
  // sgn(x) min(|x|, C|y|, C|z|) when x, y, z share a strict sign, else 0
  double sx = sgn0(x);
  if (sx != 0 && sx == sgn0(y) && sx == sgn0(z))
    return sx * S_min(S_abs(x), S_min(kPpmC * S_abs(y), kPpmC * S_abs(z)));
  return S(0.0);
}

template <class S> S d2lim4(const S& x, const S& y, const S& z, const S& t) {
  double sx = sgn0(x);
  if (sx != 0 && sx == sgn0(y) && sx == sgn0(z) && sx == sgn0(t))
    return sx * S_min(S_min(S_abs(x), kPpmC * S_abs(y)), S_min(kPpmC * S_abs(z), kPpmC * S_abs(t)));
  return S(0.0);
}

template <class S> void ppm_limit_one(const S* q, S* qm_out, S* qp_out) {
  // q[0..4] = q_{i-2..i+2}
  S qm = 7.0 / 12.0 * (q[1] + q[2]) - 1.0 / 12.0 * (q[0] + q[3]);
  S qp = 7.0 / 12.0 * (q[2] + q[3]) - 1.0 / 12.0 * (q[1] + q[4]);
  S d2m1 = q[0] - 2.0 * q[1] + q[2];
  S d20 = q[1] - 2.0 * q[2] + q[3];
  S d2p1 = q[2] - 2.0 * q[3] + q[4];
  // (3) interface limiter
  if (val((qm - q[1]) * (q[2] - qm)) < 0) {
    S d2c = 3.0 * (q[1] - 2.0 * qm + q[2]);
    qm = 0.5 * (q[1] + q[2]) - d2lim3(d2c, d2m1, d20) / 6.0;
  }
  if (val((qp - q[2]) * (q[3] - qp)) < 0) {
    S d2c = 3.0 * (q[2] - 2.0 * qp + q[3]);
    qp = 0.5 * (q[2] + q[3]) - d2lim3(d2c, d20, d2p1) / 6.0;
  }
  // (4) cell limiter
  S dqm = q[2] - qm, dqp = qp - q[2];
  if (val(dqm * dqp) <= 0 || val((q[2] - q[1]) * (q[3] - q[2])) <= 0) {
    S d2f = 6.0 * (qm - 2.0 * q[2] + qp);
    S r = S(0.0);
    if (val(d2f) != 0) r = d2lim4(d2f, d2m1, d20, d2p1) / d2f;
    qm = q[2] - r * dqm;
    qp = q[2] + r * dqp;
  } else {
    if (val(S_abs(dqm)) >= 2.0 * val(S_abs(dqp))) qm = q[2] - 2.0 * dqp;
    if (val(S_abs(dqp)) >= 2.0 * val(S_abs(dqm))) qp = q[2] + 2.0 * dqm;
  }
  *qm_out = qm;
  *qp_out = qp;
}

template <class S>
void ppmc(const Params& P, const Grid& g, const S* U, const int* p, int a, S* wl_out, S* wr_out) {
  S w[5][7], bn, tmp;
  for (int s = -2; s <= 2; ++s) dir_state(P, g, U, p, a, s, w[s + 2], s == 0 ? &bn : &tmp);
  Eigen<S> E;
  eigensystem(P.gamma, w[2], bn, E);
  // characteristic variables relative to cell i: q_s = L (W_s - W_i), so
  // q_i = 0 and the limiter's sign tests see the differences of the data
  // (projecting W_s itself and subtracting would round away differences
  // below ~1e-16 of the O(1) projected values)
  S q[5][7];
  for (int s = 0; s < 5; ++s) {
    S dw[7];
    for (int c = 0; c < 7; ++c) dw[c] = w[s][c] - w[2][c];
    matvec7(E.L, dw, q[s]);
  }
  S dm[7], dp[7];
  for (int c = 0; c < 7; ++c) {
    S col[5] = {q[0][c], q[1][c], q[2][c], q[3][c], q[4][c]};
    S qm, qp;
    ppm_limit_one(col, &qm, &qp);
    dm[c] = qm - q[2][c];
    dp[c] = qp - q[2][c];
  }
  S Wm[7], Wp[7];
  matvec7(E.R, dm, Wm);
  matvec7(E.R, dp, Wp);
  for (int c = 0; c < 7; ++c) {
    wl_out[c] = w[2][c] + Wp[c];
    wr_out[c] = w[2][c] + Wm[c];
  }
  floor_state(P, wl_out);
  floor_state(P, wr_out);
}

// face states of cell p along a: wl = W_{L, p+1/2}, wr = W_{R, p-1/2}
template <class S>
void reconstruct(const Params& P, const Grid& g, const S* U, const int* p, int a, int recon, S* wl, S* wr) {
  if (recon == 0) {
    S bn;
    dir_state(P, g, U, p, a, 0, wl, &bn);
    for (int q = 0; q < 7; ++q) wr[q] = wl[q];
  } else if (recon == 1) {
    plmc(P, g, U, p, a, wl, wr);
  } else if (recon == 3) {
    plmc(P, g, U, p, a, wl, wr, true);
  } else {
    ppmc(P, g, U, p, a, wl, wr);
  }
}

// ------------------------------------------------ Steps 2-3 / 6-7: fluxes --
// F[a][7][N]: flux through the upper a-face of each cell, solver frame of a.
// The longitudinal field is the stored face value (Sec. 2.2.3).
template <class S> void fluxes(const Params& P, const Grid& g, const S* U, int recon, S* F) {
  const long N = g.N;
  for (int a = 0; a < 3; ++a) {
    std::vector<S> WL(7 * N), WR(7 * N);
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) {
      int p[3];
      g.coords(c, p);
      S wl[7], wr[7];
      reconstruct(P, g, U, p, a, recon, wl, wr);
      for (int q = 0; q < 7; ++q) {
        WL[q * N + c] = wl[q];
        WR[q * N + c] = wr[q];
      }
    }
#pragma omp parallel for schedule(static)
    for (long c = 0; c < N; ++c) {
      int p[3];
      g.coords(c, p);
      long cn = g.shift(p, a, +1);
      S wl[7], wr[7], f[7];
      for (int q = 0; q < 7; ++q) {
        wl[q] = WL[q * N + c];
        wr[q] = WR[q * N + cn];
      }
      hlld(P.gamma, wl, wr, U[(5 + a) * N + c], f);
      for (int q = 0; q < 7; ++q) F[((long)a * 7 + q) * N + c] = f[q];
    }
  }
}

// --------------------------------------------------- O5/O6. edge EMF (CT) --
// Edge a of cell p sits at p + e_b/2 + e_c/2, (b, c) = (a+1, a+2).  Face
// fields from Table "emf": eps_a on a b-face = -F_b[B_t1], on a c-face =
// +F_c[B_t2].  Edge value: Eq. "emf-edge" with the upwinded slopes of
// Eqs. "emf-upwind-slope"/"emf-slope" (D-6: face minus reference for every
// slope; D-7: upwind by the sign of the face's mass flux, mean when zero).
// Reference field -(v x B_cc) of each cell (Sec. 2.2.4).
template <class S> S upwind(const S& mflux, const S& lo, const S& hi) {
  if (val(mflux) > 0) return lo;
  if (val(mflux) < 0) return hi;
  return 0.5 * (lo + hi);
}

template <class S> void edge_emf(const Params& P, const Grid& g, const S* U, const S* F, S* E) {
  const long N = g.N;
  std::vector<S> ref(3 * N);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < N; ++c) {
    int p[3];
    g.coords(c, p);
    Prim<S> w = primitive(P, g, U, p);
    for (int a = 0; a < 3; ++a) {
      int b = (a + 1) % 3, cc = (a + 2) % 3;
      ref[a * N + c] = -(w.v[b] * w.b[cc] - w.v[cc] * w.b[b]);
    }
  }
#pragma omp parallel for schedule(static)
  for (long c = 0; c < N; ++c) {
    int p[3];
    g.coords(c, p);
    for (int a = 0; a < 3; ++a) {
      int b = (a + 1) % 3, cc = (a + 2) % 3;
      const S* Fb = F + (long)b * 7 * N;
      const S* Fc = F + (long)cc * 7 * N;
      long q00 = c, qb = g.shift(p, b, 1), qc = g.shift(p, cc, 1), qbc = g.shift2(p, b, 1, cc, 1);
      auto bf = [&](long q) { return S(-Fb[5 * N + q]); };
      auto cf = [&](long q) { return S(Fc[6 * N + q]); };
      auto mb = [&](long q) { return Fb[q]; };
      auto mc = [&](long q) { return Fc[q]; };
      auto rf = [&](long q) { return ref[a * N + q]; };
      S avg = 0.25 * (bf(qc) + bf(q00) + cf(qb) + cf(q00));
      S Dcp = upwind(mb(qc), S(cf(q00) - rf(qc)), S(cf(qb) - rf(qbc)));
      S Dcm = upwind(mb(q00), S(cf(q00) - rf(q00)), S(cf(qb) - rf(qb)));
      S Dbp = upwind(mc(qb), S(bf(q00) - rf(qb)), S(bf(qc) - rf(qbc)));
      S Dbm = upwind(mc(q00), S(bf(q00) - rf(q00)), S(bf(qc) - rf(qc)));
      E[a * N + c] = avg + 0.25 * (Dcp + Dcm + Dbp + Dbm);
    }
  }
}

// ------------------------------------------------ O7. conservative update --
// Steps 5 and 9: U_out = U0 - h sum_a (F_a+ - F_a-)/d_a for rho, m, E (D-15:
// difference form, x then y then z) and face B_a -= h [(E_c(p) - E_c(p-e_b))/d_b
// - (E_b(p) - E_b(p-e_c))/d_c]; h = dt/2 in Step 5 (D-1), dt in Step 9.
// Index typos of the printed equations read per D-2 and D-3.
// (h is a double, or a dual number when the step size itself is differentiated)
template <class S, class H>
void update(const Params& P, const Grid& g, const S* U0, const S* F, const S* E, H h, S* Uout) {
  const long N = g.N;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < N; ++c) {
    int p[3];
    g.coords(c, p);
    for (int f = 0; f < 5; ++f) {
      S acc = U0[f * N + c];
      for (int a = 0; a < 3; ++a) {
        int comp;
        if (f == 0) comp = 0;
        else if (f == 4) comp = 4;
        else comp = 1 + ((f - 1 - a + 3) % 3);
        const S* Fa = F + ((long)a * 7 + comp) * N;
        acc = acc - (h / P.d[a]) * (Fa[c] - Fa[g.shift(p, a, -1)]);
      }
      Uout[f * N + c] = acc;
    }
    for (int a = 0; a < 3; ++a) {
      int b = (a + 1) % 3, cc = (a + 2) % 3;
      const S* Ec = E + (long)cc * N;
      const S* Eb = E + (long)b * N;
      S curl = (Ec[c] - Ec[g.shift(p, b, -1)]) / P.d[b] - (Eb[c] - Eb[g.shift(p, cc, -1)]) / P.d[cc];
      Uout[(5 + a) * N + c] = U0[(5 + a) * N + c] - h * curl;
    }
  }
}

// Floors on the conserved state after the full update (D-12): rho < rho_floor
// is raised; if the recovered P < p_floor, E is reset so that P = p_floor.
template <class S> void apply_floors(const Params& P, const Grid& g, S* U, long long* counts) {
  const long N = g.N;
  long long nr = 0, np = 0;
  for (long c = 0; c < N; ++c) {
    int p[3];
    g.coords(c, p);
    if (val(U[c]) < P.rho_floor) {
      U[c] = S(P.rho_floor);
      ++nr;
    }
    S rho = U[c];
    S m[3] = {U[N + c], U[2 * N + c], U[3 * N + c]};
    S b[3];
    for (int a = 0; a < 3; ++a) b[a] = 0.5 * (U[(5 + a) * N + g.shift(p, a, -1)] + U[(5 + a) * N + c]);
    S ke = 0.5 * (m[0] * m[0] + m[1] * m[1] + m[2] * m[2]) / rho;
    S me = 0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    S pr = (P.gamma - 1.0) * (U[4 * N + c] - ke - me);
    if (val(pr) < P.p_floor) {
      U[4 * N + c] = P.p_floor / (P.gamma - 1.0) + ke + me;
      ++np;
    }
  }
  if (counts) {
    counts[0] += nr;
    counts[1] += np;
  }
}

// ------------------------------------------------------ O11. one VL+CT step --
template <class S, class H> void step(const Params& P, S* U, H dt, long long* counts) {
  Grid g(P);
  const long N = g.N;
  std::vector<S> U0(U, U + 8 * N), Uh(8 * N), F(21 * N), E(3 * N);
  fluxes(P, g, U0.data(), 0, F.data());                       // Steps 2-3 (PCM + HLLD)
  edge_emf(P, g, U0.data(), F.data(), E.data());             // Step 4
  update(P, g, U0.data(), F.data(), E.data(), 0.5 * dt, Uh.data());  // Step 5
  fluxes(P, g, Uh.data(), P.recon, F.data());                 // Steps 6-7
  edge_emf(P, g, Uh.data(), F.data(), E.data());             // Step 8 (D-4)
  update(P, g, U0.data(), F.data(), E.data(), dt, U);        // Step 9
  apply_floors(P, g, U, counts);
}

// ----------------------------------------------------------------- O2. dt --
// Eq. dt over the cells of the box [lo, hi) (the whole grid when lo is null)
double cfl_dt(const Params& P, const double* U, double cfl, const int* lo = nullptr, const int* hi = nullptr) {
  Grid g(P);
  double best = std::numeric_limits<double>::infinity();
#pragma omp parallel for reduction(min : best) schedule(static)
  for (long c = 0; c < g.N; ++c) {
    int p[3];
    g.coords(c, p);
    if (lo && (p[0] < lo[0] || p[0] >= hi[0] || p[1] < lo[1] || p[1] >= hi[1] || p[2] < lo[2] || p[2] >= hi[2]))
      continue;
    Prim<double> w = primitive(P, g, U, p);
    for (int l = 0; l < 3; ++l) {
      int b = (l + 1) % 3, cc = (l + 2) % 3;
      double cf = fast_speed(P.gamma, w.rho, w.p, w.b[l], w.b[b], w.b[cc]);
      double t = P.d[l] / (std::fabs(w.v[l]) + cf);
      best = std::min(best, t);
    }
  }
  return cfl * best;
}

// Eq. dt with its directional derivative along dU: the minimum is taken at
// its first attaining (cell, axis) in index order, as in cfl_dt's loop, and
// differentiated there with dual numbers (one element of the subdifferential
// where cells tie).  Returns dt; *ddt receives the derivative.
double cfl_dt_jvp(const Params& P, const double* U, const double* dU, double cfl, double* ddt) {
  Grid g(P);
  double best = std::numeric_limits<double>::infinity();
  long bc = -1;
  int bl = 0;
  for (long c = 0; c < g.N; ++c) {
    int p[3];
    g.coords(c, p);
    Prim<double> w = primitive(P, g, U, p);
    for (int l = 0; l < 3; ++l) {
      double cf = fast_speed(P.gamma, w.rho, w.p, w.b[l], w.b[(l + 1) % 3], w.b[(l + 2) % 3]);
      double t = P.d[l] / (std::fabs(w.v[l]) + cf);
      if (t < best) {
        best = t;
        bc = c;
        bl = l;
      }
    }
  }
  *ddt = 0.0;
  if (bc < 0) return cfl * best;
  std::vector<Dual> X(8 * g.N);
  for (long i = 0; i < 8 * g.N; ++i) X[i] = Dual(U[i], dU[i]);
  int p[3];
  g.coords(bc, p);
  Prim<Dual> w = primitive(P, g, X.data(), p);
  Dual cf = fast_speed(P.gamma, w.rho, w.p, w.b[bl], w.b[(bl + 1) % 3], w.b[(bl + 2) % 3]);
  Dual t = P.d[bl] / (S_abs(w.v[bl]) + cf);
  *ddt = cfl * t.d;
  return cfl * best;
}

}  // namespace

// ======================================================= extern "C" API ====
extern "C" {

void oracle_primitives(const Params* P, const double* U, double* W) {
  Grid g(*P);
  for (long c = 0; c < g.N; ++c) {
    int p[3];
    g.coords(c, p);
    Prim<double> w = primitive(*P, g, U, p);
    double out[8] = {w.rho, w.v[0], w.v[1], w.v[2], w.p, w.b[0], w.b[1], w.b[2]};
    for (int f = 0; f < 8; ++f) W[f * g.N + c] = out[f];
  }
}

double oracle_dt(const Params* P, const double* U, double cfl) { return cfl_dt(*P, U, cfl); }

// threads of the OpenMP loops (for timing the oracle single-threaded); returns the previous count
int oracle_set_threads(int n) {
#ifdef _OPENMP
  const int prev = omp_get_max_threads();
  if (n > 0) omp_set_num_threads(n);
  return prev;
#else
  (void)n;
  return 1;
#endif
}

double oracle_dt_box(const Params* P, const double* U, double cfl, const int* lo, const int* hi) {
  return cfl_dt(*P, U, cfl, lo, hi);
}

double oracle_fast_speed(double gamma, double rho, double p, double bl, double bt1, double bt2) {
  return fast_speed(gamma, rho, p, bl, bt1, bt2);
}

void oracle_hlld(double gamma, const double* wl, const double* wr, double bn, double* f) {
  hlld(gamma, wl, wr, bn, f);
}

// speeds[5] = SL, S*L, SM, S*R, SR; states[6][7] = UL, U*L, U**L, U**R, U*R, UR;
// fl[2][7] = F(UL), F(UR).  Returns 1 if star states were formed.
int oracle_hlld_detail(double gamma, const double* wl, const double* wr, double bn, double* f, double* speeds,
                       double* states, double* fl) {
  HlldDetail<double> d;
  hlld(gamma, wl, wr, bn, f, &d);
  speeds[0] = d.SL;
  speeds[4] = d.SR;
  if (d.star) {
    speeds[1] = d.SsL;
    speeds[2] = d.SM;
    speeds[3] = d.SsR;
  }
  for (int q = 0; q < 7; ++q) {
    states[0 * 7 + q] = d.UL[q];
    states[5 * 7 + q] = d.UR[q];
    fl[q] = d.FL[q];
    fl[7 + q] = d.FR[q];
    if (d.star) {
      states[1 * 7 + q] = d.UsL[q];
      states[2 * 7 + q] = d.UssL[q];
      states[3 * 7 + q] = d.UssR[q];
      states[4 * 7 + q] = d.UsR[q];
    }
  }
  return d.star ? 1 : 0;
}

void oracle_eigen(double gamma, const double* w, double bn, double* lam, double* R, double* L) {
  Eigen<double> E;
  eigensystem(gamma, w, bn, E);
  for (int i = 0; i < 7; ++i) {
    lam[i] = E.lam[i];
    for (int j = 0; j < 7; ++j) {
      R[i * 7 + j] = E.R[i][j];
      L[i * 7 + j] = E.L[i][j];
    }
  }
}

// WL[7][N] = W_{L, p+1/2}, WR[7][N] = W_{R, p-1/2} of every cell p along axis a.
// recon: 0 PCM, 1 PLMC, 2 PPMC, 3 PLM with primitive limiting.
void oracle_recon(const Params* P, const double* U, int a, int recon, double* WL, double* WR) {
  Grid g(*P);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < g.N; ++c) {
    int p[3];
    g.coords(c, p);
    double wl[7], wr[7];
    reconstruct(*P, g, U, p, a, recon, wl, wr);
    for (int q = 0; q < 7; ++q) {
      WL[q * g.N + c] = wl[q];
      WR[q * g.N + c] = wr[q];
    }
  }
}

void oracle_fluxes(const Params* P, const double* U, int recon, double* F) {
  Grid g(*P);
  fluxes(*P, g, U, recon, F);
}

void oracle_edges(const Params* P, const double* U, const double* F, double* E) {
  Grid g(*P);
  edge_emf(*P, g, U, F, E);
}

void oracle_update(const Params* P, const double* U0, const double* F, const double* E, double h, double* Uout) {
  Grid g(*P);
  update(*P, g, U0, F, E, h, Uout);
}

void oracle_step(const Params* P, double* U, double dt, long long* counts) { step(*P, U, dt, counts); }

// Jacobian-vector product of one step at fixed dt: U -> U^{n+1}, dU -> J dU.
void oracle_step_jvp(const Params* P, double* U, double* dU, double dt) {
  Grid g(*P);
  const long M = 8 * g.N;
  std::vector<Dual> X(M);
  for (long i = 0; i < M; ++i) X[i] = Dual(U[i], dU[i]);
  step(*P, X.data(), dt, nullptr);
  for (long i = 0; i < M; ++i) {
    U[i] = X[i].v;
    dU[i] = X[i].d;
  }
}

// Jacobian-vector product of one step at the CFL dt of its start state:
// U^{n+1} = step(U, dt(U)), so J dU = (dstep/dU) dU + (dstep/d dt) (d dt/dU) dU.
// *dt_out receives dt.
void oracle_step_cfl_jvp(const Params* P, double* U, double* dU, double cfl, double* dt_out) {
  Grid g(*P);
  double ddt = 0.0;
  const double dt = cfl_dt_jvp(*P, U, dU, cfl, &ddt);
  const long M = 8 * g.N;
  std::vector<Dual> X(M);
  for (long i = 0; i < M; ++i) X[i] = Dual(U[i], dU[i]);
  step(*P, X.data(), Dual(dt, ddt), nullptr);
  for (long i = 0; i < M; ++i) {
    U[i] = X[i].v;
    dU[i] = X[i].d;
  }
  *dt_out = dt;
}

double oracle_dt_jvp(const Params* P, const double* U, const double* dU, double cfl, double* ddt) {
  return cfl_dt_jvp(*P, U, dU, cfl, ddt);
}

// Forward-mode derivative of the HLLD flux: f = HLLD(wl, wr, bn), df = J (dwl, dwr, dbn).
void oracle_hlld_jvp(double gamma, const double* wl, const double* wr, double bn, const double* dwl,
                     const double* dwr, double dbn, double* f, double* df) {
  Dual a[7], b[7], out[7];
  for (int q = 0; q < 7; ++q) {
    a[q] = Dual(wl[q], dwl[q]);
    b[q] = Dual(wr[q], dwr[q]);
  }
  hlld(gamma, a, b, Dual(bn, dbn), out);
  for (int q = 0; q < 7; ++q) {
    f[q] = out[q].v;
    df[q] = out[q].d;
  }
}

// Forward-mode derivative of U -> (W_L, W_R) along axis a (primitives then
// reconstruction): WL, WR, dWL, dWR are [7][N].
void oracle_recon_jvp(const Params* P, const double* U, const double* dU, int a, int recon, double* WL, double* WR,
                      double* dWL, double* dWR) {
  Grid g(*P);
  const long N = g.N;
  std::vector<Dual> X(8 * N);
  for (long i = 0; i < 8 * N; ++i) X[i] = Dual(U[i], dU[i]);
#pragma omp parallel for schedule(static)
  for (long c = 0; c < N; ++c) {
    int p[3];
    g.coords(c, p);
    Dual wl[7], wr[7];
    reconstruct(*P, g, X.data(), p, a, recon, wl, wr);
    for (int q = 0; q < 7; ++q) {
      WL[q * N + c] = wl[q].v;
      dWL[q * N + c] = wl[q].d;
      WR[q * N + c] = wr[q].v;
      dWR[q * N + c] = wr[q].d;
    }
  }
}

// max |div B| (face differences, per cell) and plain sums of the 8 fields.
void oracle_diagnostics(const Params* P, const double* U, double* divb_max, double* totals) {
  Grid g(*P);
  const long N = g.N;
  double m = 0;
  for (long c = 0; c < N; ++c) {
    int p[3];
    g.coords(c, p);
    double dv = 0;
    for (int a = 0; a < 3; ++a) dv += (U[(5 + a) * N + c] - U[(5 + a) * N + g.shift(p, a, -1)]) / P->d[a];
    m = std::max(m, std::fabs(dv));
  }
  *divb_max = m;
  for (int f = 0; f < 8; ++f) {
    long double s = 0;
    for (long c = 0; c < N; ++c) s += U[f * N + c];
    totals[f] = (double)s;
  }
}

}  // extern "C"
