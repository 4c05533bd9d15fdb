// sanitize_check.cpp -- runs every entry point of the oracle once on small
// ragged periodic grids and random face states, for a build of the oracle
// with -fsanitize=address,undefined (tests/test_oracle_sanitize.py).  Test
// infrastructure, like the oracle itself: exits 0 when every output is
// finite, 1 otherwise; the sanitizers abort on any out-of-bounds access or
// undefined behaviour.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

// layout of the oracle's Params (mhd_oracle.cpp)
struct OParams {
  int n[3];
  double d[3];
  double gamma;
  double rho_floor, p_floor;
  int recon;
};

extern "C" {
void oracle_primitives(const OParams* P, const double* U, double* W);
double oracle_dt(const OParams* P, const double* U, double cfl);
double oracle_dt_box(const OParams* P, const double* U, double cfl, const int* lo, const int* hi);
double oracle_fast_speed(double gamma, double rho, double p, double bl, double bt1, double bt2);
void oracle_hlld(double gamma, const double* wl, const double* wr, double bn, double* f);
int oracle_hlld_detail(double gamma, const double* wl, const double* wr, double bn, double* f, double* speeds,
                       double* states, double* fl);
void oracle_eigen(double gamma, const double* w, double bn, double* lam, double* R, double* L);
void oracle_recon(const OParams* P, const double* U, int a, int recon, double* WL, double* WR);
void oracle_fluxes(const OParams* P, const double* U, int recon, double* F);
void oracle_edges(const OParams* P, const double* U, const double* F, double* E);
void oracle_update(const OParams* P, const double* U0, const double* F, const double* E, double h, double* Uout);
void oracle_step(const OParams* P, double* U, double dt, long long* counts);
void oracle_step_jvp(const OParams* P, double* U, double* dU, double dt);
void oracle_step_cfl_jvp(const OParams* P, double* U, double* dU, double cfl, double* dt_out);
double oracle_dt_jvp(const OParams* P, const double* U, const double* dU, double cfl, double* ddt);
void oracle_hlld_jvp(double gamma, const double* wl, const double* wr, double bn, const double* dwl,
                     const double* dwr, double dbn, double* f, double* df);
void oracle_recon_jvp(const OParams* P, const double* U, const double* dU, int a, int recon, double* WL, double* WR,
                      double* dWL, double* dWR);
void oracle_diagnostics(const OParams* P, const double* U, double* divb_max, double* totals);
}

namespace {

std::mt19937_64 rng(7);
double uni(double a, double b) { return std::uniform_real_distribution<double>(a, b)(rng); }

bool finite_all(const std::vector<double>& v) {
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

// a valid state: rho, P > 0 and random velocities and face fields
std::vector<double> state(const OParams& P, double gamma) {
  const int nx = P.n[0], ny = P.n[1], nz = P.n[2];
  const long N = (long)nx * ny * nz;
  std::vector<double> U(8 * N);
  for (long c = 0; c < N; ++c) {
    U[5 * N + c] = 0.5 + uni(-0.2, 0.2);
    U[6 * N + c] = uni(-0.3, 0.3);
    U[7 * N + c] = uni(-0.3, 0.3);
  }
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const long c = ((long)k * ny + j) * nx + i;
        const long cx = ((long)k * ny + j) * nx + (i + nx - 1) % nx;
        const long cy = ((long)k * ny + (j + ny - 1) % ny) * nx + i;
        const long cz = ((long)((k + nz - 1) % nz) * ny + j) * nx + i;
        const double b[3] = {0.5 * (U[5 * N + c] + U[5 * N + cx]), 0.5 * (U[6 * N + c] + U[6 * N + cy]),
                             0.5 * (U[7 * N + c] + U[7 * N + cz])};
        const double rho = uni(0.8, 1.2), p = uni(0.8, 1.2);
        const double v[3] = {uni(-0.5, 0.5), uni(-0.5, 0.5), uni(-0.5, 0.5)};
        U[c] = rho;
        for (int a = 0; a < 3; ++a) U[(1 + a) * N + c] = rho * v[a];
        U[4 * N + c] = p / (gamma - 1.0) + 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) +
                       0.5 * (b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
      }
  return U;
}

bool grid_case(int nx, int ny, int nz, int recon) {
  const double gamma = 5.0 / 3.0;
  OParams P{{nx, ny, nz}, {1.0 / nx, 1.0 / ny, 1.0 / nz}, gamma, 1e-20, 1e-20, recon};
  const long N = (long)nx * ny * nz;
  std::vector<double> U = state(P, gamma), W(8 * N), F(21 * N), E(3 * N), V(8 * N);
  bool ok = true;
  oracle_primitives(&P, U.data(), W.data());
  const double dt = oracle_dt(&P, U.data(), 0.3);
  const int lo[3] = {1, 1, 1}, hi[3] = {nx - 1, ny - 1, nz - 1};
  ok &= std::isfinite(dt) && std::isfinite(oracle_dt_box(&P, U.data(), 0.3, lo, hi));
  oracle_fluxes(&P, U.data(), recon, F.data());
  oracle_edges(&P, U.data(), F.data(), E.data());
  oracle_update(&P, U.data(), F.data(), E.data(), 0.5 * dt, V.data());
  ok &= finite_all(W) && finite_all(F) && finite_all(E) && finite_all(V);
  std::vector<double> S = U;
  long long counts[2] = {0, 0};
  oracle_step(&P, S.data(), dt, counts);
  double divb = 0, totals[8];
  oracle_diagnostics(&P, S.data(), &divb, totals);
  ok &= finite_all(S) && std::isfinite(divb);
  std::vector<double> WL(7 * N), WR(7 * N), dWL(7 * N), dWR(7 * N), dU(8 * N);
  for (double& x : dU) x = uni(-1e-3, 1e-3);
  for (int a = 0; a < 3; ++a) {
    oracle_recon(&P, U.data(), a, recon, WL.data(), WR.data());
    ok &= finite_all(WL) && finite_all(WR);
  }
  if (recon != 3) {  // the variant without a derivative path
    for (int a = 0; a < 3; ++a) {
      oracle_recon_jvp(&P, U.data(), dU.data(), a, recon, WL.data(), WR.data(), dWL.data(), dWR.data());
      ok &= finite_all(dWL) && finite_all(dWR);
    }
    std::vector<double> J = U, dJ = dU;
    oracle_step_jvp(&P, J.data(), dJ.data(), dt);
    ok &= finite_all(J) && finite_all(dJ);
    J = U;
    dJ = dU;
    double dtc = 0, ddt = 0;
    oracle_step_cfl_jvp(&P, J.data(), dJ.data(), 0.3, &dtc);
    ok &= finite_all(J) && finite_all(dJ) && std::isfinite(oracle_dt_jvp(&P, U.data(), dU.data(), 0.3, &ddt));
  }
  return ok;
}

bool riemann_cases() {
  bool ok = true;
  const double gamma = 5.0 / 3.0;
  for (int t = 0; t < 200; ++t) {
    double wl[7], wr[7], dwl[7], dwr[7], f[7], df[7], speeds[5], states[42], fl[14], lam[7], R[49], L[49];
    for (int q = 0; q < 7; ++q) {
      wl[q] = uni(-1.0, 1.0);
      wr[q] = uni(-1.0, 1.0);
      dwl[q] = uni(-1.0, 1.0);
      dwr[q] = uni(-1.0, 1.0);
    }
    wl[0] = uni(0.2, 2.0), wr[0] = uni(0.2, 2.0), wl[4] = uni(0.2, 2.0), wr[4] = uni(0.2, 2.0);
    if (t % 4 == 1) wl[5] = wl[6] = wr[5] = wr[6] = 0.0;  // no transverse field
    const double bn = t % 4 == 2 ? 0.0 : uni(-1.0, 1.0);  // no normal field
    oracle_hlld(gamma, wl, wr, bn, f);
    oracle_hlld_detail(gamma, wl, wr, bn, f, speeds, states, fl);
    oracle_hlld_jvp(gamma, wl, wr, bn, dwl, dwr, 0.5, f, df);
    oracle_eigen(gamma, wl, bn, lam, R, L);
    ok &= std::isfinite(oracle_fast_speed(gamma, wl[0], wl[4], bn, wl[5], wl[6]));
    for (int q = 0; q < 7; ++q) ok &= std::isfinite(f[q]) && std::isfinite(df[q]) && std::isfinite(lam[q]);
    for (int q = 0; q < 49; ++q) ok &= std::isfinite(R[q]) && std::isfinite(L[q]);
  }
  return ok;
}

}  // namespace

int main() {
  bool ok = riemann_cases();
  const int sizes[3][3] = {{7, 5, 6}, {4, 9, 5}, {11, 4, 4}};
  for (const auto& s : sizes)
    for (int recon = 0; recon <= 3; ++recon) {
      const bool r = grid_case(s[0], s[1], s[2], recon);
      if (!r) std::printf("non-finite output: %d x %d x %d, recon %d\n", s[0], s[1], s[2], recon);
      ok &= r;
    }
  std::printf(ok ? "ok\n" : "FAILED\n");
  return ok ? 0 : 1;
}
