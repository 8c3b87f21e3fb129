// Host-side consistency checks of the CUDA path's element routines (the header
// is plain C++ outside nvcc), on seeded random elements, parameters, gravity
// directions and element sources:
//   J v      against central differences of the element residual,
//   J^T w    against the transpose of the 40 columns of J,
//   diag(J)  against those columns' diagonal,
//   J v from the linearisation store against J v,
//   the design sensitivity w^T dr/dgamma against central differences in gamma.
// Prints the largest relative error of each check; exit status 1 if any is
// above its bound (1e-12 for the exact identities, 1e-6 for the differences).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>

#include "../../paper_1508_04596_gb300/csrc/nc_element.cuh"

using namespace nc;
typedef double M[5][8];

static double maxabs(const M a) {
  double m = 0.0;
  for (int f = 0; f < 5; ++f)
    for (int a2 = 0; a2 < 8; ++a2) m = std::fmax(m, std::fabs(a[f][a2]));
  return m;
}

int main() {
  std::mt19937_64 rng(7741);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  const double eg[3][3] = {{0.0, 0.0, -1.0}, {0.0, -1.0, 0.0}, {0.6, 0.0, -0.8}};
  double e_fd = 0.0, e_tr = 0.0, e_diag = 0.0, e_lin = 0.0, e_sens = 0.0;
  for (int trial = 0; trial < 16; ++trial) {
    const double h = 1.0 / (4 + 5 * trial);
    const ElemConst<double> c =
        make_const<double>(h, std::pow(10.0, 2 + trial % 5), trial % 2 ? 1.0 : 0.71,
                           1e4 * (1 + trial % 3), 1.0 + trial % 4, 0.5 + trial % 3,
                           trial % 2 ? 0.1 : 0.01, eg[trial % 3]);
    M xe;
    for (int f = 0; f < 5; ++f)
      for (int a = 0; a < 8; ++a) xe[f][a] = U(rng) * (f == 3 ? 20.0 : 1.0);
    const double gam = 0.5 + 0.45 * U(rng);
    const double s = trial % 2 ? 0.0 : 3.0 * (1.0 + U(rng));
    // the 40 columns of J_e
    double J[40][40];  // J[row f*8+a][col g*8+b]
    for (int col = 0; col < 40; ++col) {
      M ve = {}, out;
      ve[col / 8][col % 8] = 1.0;
      elem_jvp<double>(xe, ve, gam, s, c, out);
      for (int f = 0; f < 5; ++f)
        for (int a = 0; a < 8; ++a) J[f * 8 + a][col] = out[f][a];
    }
    // J v against central differences of the residual
    M v;
    for (int f = 0; f < 5; ++f)
      for (int a = 0; a < 8; ++a) v[f][a] = U(rng) * (f == 3 ? 20.0 : 1.0);
    const double eps = 1e-6;
    M xp, xm, rp, rm, jv;
    for (int f = 0; f < 5; ++f)
      for (int a = 0; a < 8; ++a) {
        xp[f][a] = xe[f][a] + eps * v[f][a];
        xm[f][a] = xe[f][a] - eps * v[f][a];
      }
    elem_residual<double>(xp, gam, s, c, rp);
    elem_residual<double>(xm, gam, s, c, rm);
    elem_jvp<double>(xe, v, gam, s, c, jv);
    M fd;
    for (int f = 0; f < 5; ++f)
      for (int a = 0; a < 8; ++a) fd[f][a] = (rp[f][a] - rm[f][a]) / (2.0 * eps) - jv[f][a];
    e_fd = std::fmax(e_fd, maxabs(fd) / maxabs(jv));
    // J^T w against the columns
    M w, jtw, d;
    for (int f = 0; f < 5; ++f)
      for (int a = 0; a < 8; ++a) w[f][a] = U(rng);
    elem_jtvp<double>(xe, w, gam, s, c, jtw);
    for (int col = 0; col < 40; ++col) {
      double acc = 0.0;
      for (int row = 0; row < 40; ++row) acc += J[row][col] * w[row / 8][row % 8];
      d[col / 8][col % 8] = jtw[col / 8][col % 8] - acc;
    }
    e_tr = std::fmax(e_tr, maxabs(d) / maxabs(jtw));
    // diag(J)
    M dg;
    elem_diag<double>(xe, gam, s, c, dg);
    double dmax = 0.0, derr = 0.0;
    for (int i = 0; i < 40; ++i) {
      dmax = std::fmax(dmax, std::fabs(J[i][i]));
      derr = std::fmax(derr, std::fabs(dg[i / 8][i % 8] - J[i][i]));
    }
    e_diag = std::fmax(e_diag, derr / dmax);
    // J v from the linearisation store
    double cache[LIN_SLOTS];
    elem_linearize<double>(xe, gam, s, c, cache, 1);
    double ue[3][8];
    std::memcpy(ue, xe, sizeof(ue));
    M jvl, dl;
    elem_jvp_lin<double>(cache, 1, ue, v, gam, s, c, jvl);
    for (int f = 0; f < 5; ++f)
      for (int a = 0; a < 8; ++a) dl[f][a] = jvl[f][a] - jv[f][a];
    e_lin = std::fmax(e_lin, maxabs(dl) / maxabs(jv));
    // w^T dr/dgamma against central differences in gamma
    const double sens = elem_sens<double>(xe, w, gam, s, c);
    const double eg2 = 1e-6;
    M gp, gm;
    elem_residual<double>(xe, gam + eg2, s, c, gp);
    elem_residual<double>(xe, gam - eg2, s, c, gm);
    double fdg = 0.0, scale = 0.0;
    for (int f = 0; f < 5; ++f)
      for (int a = 0; a < 8; ++a) {
        const double t = w[f][a] * (gp[f][a] - gm[f][a]) / (2.0 * eg2);
        fdg += t;
        scale += std::fabs(t);
      }
    e_sens = std::fmax(e_sens, std::fabs(sens - fdg) / std::fmax(scale, 1e-300));
  }
  std::printf("jvp_fd %.3e jtvp %.3e diag %.3e jvp_lin %.3e sens_fd %.3e\n", e_fd, e_tr, e_diag,
              e_lin, e_sens);
  const bool ok = e_fd <= 1e-6 && e_tr <= 1e-12 && e_diag <= 1e-12 && e_lin <= 1e-12 &&
                  e_sens <= 1e-6;
  return ok ? 0 : 1;
}
