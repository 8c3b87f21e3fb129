// Host-side check of the packed-pair FP32 element products (nc_element_f2.cuh,
// plain C++ outside nvcc): elem_jvp_f2 and elem_jtvp_f2 against the scalar
// elem_jvp / elem_jtvp, in FP32 and in FP64 on the same inputs, on seeded random
// elements, parameters, gravity directions and element sources.  The packed
// routines reorder some FP32 sums, so they agree with the FP32 scalar routines to
// FP32 rounding, and with the FP64 ones as closely as the FP32 scalar ones do.
// Prints the largest errors (relative to the largest output); exit status 1 if
// any is above 1e-5.
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_1508_04596_gb300/csrc/nc_element_f2.cuh"

using namespace nc;

template <typename A, typename B>
static double relmax(const A a[5][8], const B b[5][8]) {
  double m = 0.0, s = 0.0;
  for (int f = 0; f < 5; ++f)
    for (int k = 0; k < 8; ++k) {
      m = std::fmax(m, std::fabs((double)a[f][k] - (double)b[f][k]));
      s = std::fmax(s, std::fabs((double)b[f][k]));
    }
  return m / s;
}

int main() {
  std::mt19937_64 rng(9127);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  const double eg[3][3] = {{0.0, 0.0, -1.0}, {0.0, -1.0, 0.0}, {0.6, 0.0, -0.8}};
  double e32[2] = {0.0, 0.0}, e64[2] = {0.0, 0.0}, s64[2] = {0.0, 0.0};
  for (int trial = 0; trial < 64; ++trial) {
    const double h = 1.0 / (4 + 5 * (trial % 16));
    const double Gr = std::pow(10.0, 2 + trial % 5), Pr = trial % 2 ? 1.0 : 0.71;
    const double amax = 1e4 * (1 + trial % 3), qa = 1.0 + trial % 4, qf = 0.5 + trial % 3;
    const double Ck = trial % 2 ? 0.1 : 0.01;
    const ElemConst<float> cf = make_const<float>(h, Gr, Pr, amax, qa, qf, Ck, eg[trial % 3]);
    const ElemConst<double> cd = make_const<double>(h, Gr, Pr, amax, qa, qf, Ck, eg[trial % 3]);
    float xf[5][8], vf[5][8];
    double xd[5][8], vd[5][8];
    for (int f = 0; f < 5; ++f)
      for (int a = 0; a < 8; ++a) {
        xf[f][a] = (float)(U(rng) * (f == 3 ? 20.0 : 1.0));
        vf[f][a] = (float)(U(rng) * (f == 3 ? 20.0 : 1.0));
        xd[f][a] = xf[f][a];
        vd[f][a] = vf[f][a];
      }
    const float gam = (float)(0.5 + 0.45 * U(rng));
    const float s = trial % 2 ? 0.0f : (float)(3.0 * (1.0 + U(rng)));
    for (int tr = 0; tr < 2; ++tr) {
      float o2[5][8], o1[5][8];
      double od[5][8];
      if (tr) {
        elem_jtvp_f2(xf, vf, gam, s, cf, o2);
        elem_jtvp<float>(xf, vf, gam, s, cf, o1);
        elem_jtvp<double>(xd, vd, (double)gam, (double)s, cd, od);
      } else {
        elem_jvp_f2(xf, vf, gam, s, cf, o2);
        elem_jvp<float>(xf, vf, gam, s, cf, o1);
        elem_jvp<double>(xd, vd, (double)gam, (double)s, cd, od);
      }
      e32[tr] = std::fmax(e32[tr], relmax(o2, o1));
      e64[tr] = std::fmax(e64[tr], relmax(o2, od));
      s64[tr] = std::fmax(s64[tr], relmax(o1, od));
    }
  }
  std::printf("J v   : packed vs FP32 %.2e, packed vs FP64 %.2e (FP32 scalar vs FP64 %.2e)\n",
              e32[0], e64[0], s64[0]);
  std::printf("J^T w : packed vs FP32 %.2e, packed vs FP64 %.2e (FP32 scalar vs FP64 %.2e)\n",
              e32[1], e64[1], s64[1]);
  const bool ok = e32[0] <= 1e-5 && e32[1] <= 1e-5 && e64[0] <= 1e-5 && e64[1] <= 1e-5;
  return ok ? 0 : 1;
}
