// Prints the CUDA path's element rows (nc_element.cuh built as plain C++) for
// elements read from standard input, so that a test can compare them with the
// oracle's element residual and its complex-step Jacobian.  Per element, input:
//   h Gr Pr alpha_max q_alpha q_f Ck eg0 eg1 eg2 gamma s
//   x[a][f] for a = 0..7, f = 0..4 (40 values), then v[a][f] (40 values)
// output (one line each, in the order (a, f)): the residual rows, J v, J^T v
// (FP64), then J v and J^T v of the FP32 packed-pair routines.
#include <cstdio>

#include "../../paper_1508_04596_gb300/csrc/nc_element_f2.cuh"

using namespace nc;

static void put(const double o[5][8]) {
  for (int a = 0; a < 8; ++a)
    for (int f = 0; f < 5; ++f) std::printf("%.17g ", o[f][a]);
  std::printf("\n");
}
static void putf(const float o[5][8]) {
  for (int a = 0; a < 8; ++a)
    for (int f = 0; f < 5; ++f) std::printf("%.9g ", (double)o[f][a]);
  std::printf("\n");
}

int main() {
  double h, Gr, Pr, am, qa, qf, Ck, eg[3], gam, s;
  while (std::scanf("%lf %lf %lf %lf %lf %lf %lf %lf %lf %lf %lf %lf", &h, &Gr, &Pr, &am, &qa,
                    &qf, &Ck, &eg[0], &eg[1], &eg[2], &gam, &s) == 12) {
    double x[5][8], v[5][8], o[5][8];
    float xf[5][8], vf[5][8], of[5][8];
    for (int a = 0; a < 8; ++a)
      for (int f = 0; f < 5; ++f)
        if (std::scanf("%lf", &x[f][a]) != 1) return 2;
    for (int a = 0; a < 8; ++a)
      for (int f = 0; f < 5; ++f)
        if (std::scanf("%lf", &v[f][a]) != 1) return 2;
    for (int f = 0; f < 5; ++f)
      for (int a = 0; a < 8; ++a) {
        xf[f][a] = (float)x[f][a];
        vf[f][a] = (float)v[f][a];
      }
    const ElemConst<double> c = make_const<double>(h, Gr, Pr, am, qa, qf, Ck, eg);
    const ElemConst<float> cf = make_const<float>(h, Gr, Pr, am, qa, qf, Ck, eg);
    elem_residual<double>(x, gam, s, c, o);
    put(o);
    elem_jvp<double>(x, v, gam, s, c, o);
    put(o);
    elem_jtvp<double>(x, v, gam, s, c, o);
    put(o);
    elem_jvp_f2(xf, vf, (float)gam, (float)s, cf, of);
    putf(of);
    elem_jtvp_f2(xf, vf, (float)gam, (float)s, cf, of);
    putf(of);
  }
  return 0;
}
