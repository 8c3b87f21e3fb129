// Host-side consistency check of the element routines of the CUDA path (the
// header is plain C++ outside nvcc): every column of the element Jacobian from
// elem_column_lin (unit direction written out, nonzero tangent terms only)
// against the general products elem_jvp_lin (from the linearisation store) and
// elem_jvp (re-interpolating the state) with the same unit direction, on
// seeded random elements, parameters and element sources.  Prints the largest
// relative difference; exit status 1 above 1e-12.
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_1508_04596_gb300/csrc/nc_element.cuh"

using namespace nc;

template <int G>
static void column(const double* cache, double ub, int b, double gam, double s,
                   const ElemConst<double>& c, double out[5][8]) {
  elem_column_lin<double, G>(cache, 1, ub, b, gam, s, c, out);
}

int main() {
  std::mt19937_64 rng(20240611);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  const double eg[3][3] = {{0.0, 0.0, -1.0}, {0.0, -1.0, 0.0}, {0.6, 0.0, -0.8}};
  double worst = 0.0;
  for (int trial = 0; trial < 24; ++trial) {
    const double h = 1.0 / (4 + 3 * trial);
    const double Gr = std::pow(10.0, 2 + trial % 5);
    const ElemConst<double> c =
        make_const<double>(h, Gr, trial % 2 ? 1.0 : 0.71, 1e4 * (1 + trial % 3), 1.0 + trial % 4,
                           0.5 + trial % 3, 0.1, eg[trial % 3]);
    double xe[5][8];
    for (int f = 0; f < 5; ++f)
      for (int a = 0; a < 8; ++a) xe[f][a] = U(rng) * (f == 3 ? 50.0 : (trial % 4 == 0 ? 1e-3 : 1.0));
    const double gam = 0.5 + 0.5 * U(rng);
    const double s = trial % 2 ? 0.0 : 1e4 * (0.5 + 0.5 * U(rng));
    double cache[LIN_SLOTS];
    elem_linearize<double>(xe, gam, s, c, cache, 1);
    double ue[3][8];
    for (int i = 0; i < 3; ++i)
      for (int a = 0; a < 8; ++a) ue[i][a] = xe[i][a];
    for (int col = 0; col < 40; ++col) {
      const int b = col / 5, g = col % 5;
      double ve[5][8] = {};
      ve[g][b] = 1.0;
      double ref[5][8], ref2[5][8], got[5][8];
      elem_jvp_lin<double>(cache, 1, ue, ve, gam, s, c, ref);
      elem_jvp<double>(xe, ve, gam, s, c, ref2);
      const double ub = g < 3 ? xe[g][b] : 0.0;
      switch (g) {
        case 0: column<0>(cache, ub, b, gam, s, c, got); break;
        case 1: column<1>(cache, ub, b, gam, s, c, got); break;
        case 2: column<2>(cache, ub, b, gam, s, c, got); break;
        case 3: column<3>(cache, ub, b, gam, s, c, got); break;
        default: column<4>(cache, ub, b, gam, s, c, got);
      }
      double scale = 0.0, d1 = 0.0, d2 = 0.0;
      for (int f = 0; f < 5; ++f)
        for (int a = 0; a < 8; ++a) {
          scale = std::fmax(scale, std::fabs(ref[f][a]));
          d1 = std::fmax(d1, std::fabs(got[f][a] - ref[f][a]));
          d2 = std::fmax(d2, std::fabs(got[f][a] - ref2[f][a]));
        }
      if (scale == 0.0) {
        std::printf("column %d of trial %d is zero\n", col, trial);
        return 1;
      }
      worst = std::fmax(worst, std::fmax(d1, d2) / scale);
    }
  }
  std::printf("%.3e\n", worst);
  return worst <= 1e-12 ? 0 : 1;
}
