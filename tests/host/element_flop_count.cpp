// Arithmetic operation counts of the CUDA path's element routines, per element:
// the routines of nc_element.cuh instantiated with a number type that counts
// every +, -, * and / (one flop each, so an FMA counts 2) and every reciprocal
// square root (one flop), with unary minus free.  These are the algorithmic
// flop figures the benchmark's ALU roofline divides by the measured time.
//
// Prints one line "name count" per routine:
//   residual  r_e(x_e)                               (elem_residual)
//   jvp       J_e v_e re-interpolating the state     (elem_jvp)
//   jtvp      J_e^T w_e                              (elem_jtvp)
//   diag      diag(J_e)                              (elem_diag)
//   sens      lambda_e^T dr_e/dgamma_e               (elem_sens)
//   linearize the linearisation store of one element (elem_linearize)
//   jvp_lin   J_e v_e from the store                 (elem_jvp_lin)
//   jtvp_lin  J_e^T w_e from the store               (elem_jtvp_lin)
// The counts do not depend on the values (the routines have no data-dependent
// branches), so one seeded element suffices.
#include <cmath>
#include <cstdio>

namespace cnt {
long long ops = 0;
struct N {
  double v;
  N() : v(0.0) {}
  N(double x) : v(x) {}
};
inline N operator+(N a, N b) { ++ops; return N(a.v + b.v); }
inline N operator-(N a, N b) { ++ops; return N(a.v - b.v); }
inline N operator*(N a, N b) { ++ops; return N(a.v * b.v); }
inline N operator/(N a, N b) { ++ops; return N(a.v / b.v); }
inline N operator-(N a) { return N(-a.v); }
inline N& operator+=(N& a, N b) { a = a + b; return a; }
inline N& operator-=(N& a, N b) { a = a - b; return a; }
inline N& operator*=(N& a, N b) { a = a * b; return a; }
}  // namespace cnt

#include "../../paper_1508_04596_gb300/csrc/nc_element.cuh"

namespace nc {
template <>
inline cnt::N nc_rsqrt<cnt::N>(cnt::N v) {
  ++cnt::ops;
  return cnt::N(1.0 / std::sqrt(v.v));
}
}  // namespace nc

using nc::ElemConst;
using cnt::N;

int main() {
  const double eg[3] = {0.0, 0.0, -1.0};
  const ElemConst<N> c = nc::make_const<N>(1.0 / 64, 1e4, 0.71, 1e4, 1.0, 1.0, 0.1, eg);
  N xe[5][8], ve[5][8], out[5][8], ue[3][8];
  for (int f = 0; f < 5; ++f)
    for (int a = 0; a < 8; ++a) {
      xe[f][a] = N(0.1 * (f + 1) + 0.01 * a);
      ve[f][a] = N(0.2 * (f + 1) - 0.03 * a);
    }
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 8; ++a) ue[i][a] = xe[i][a];
  const N gam(0.4), s(2.0);
  N cache[nc::LIN_SLOTS];
  long long n;

  cnt::ops = 0;
  nc::elem_residual<N>(xe, gam, s, c, out);
  std::printf("residual %lld\n", cnt::ops);
  cnt::ops = 0;
  nc::elem_jvp<N>(xe, ve, gam, s, c, out);
  std::printf("jvp %lld\n", cnt::ops);
  cnt::ops = 0;
  nc::elem_jtvp<N>(xe, ve, gam, s, c, out);
  std::printf("jtvp %lld\n", cnt::ops);
  cnt::ops = 0;
  nc::elem_diag<N>(xe, gam, s, c, out);
  std::printf("diag %lld\n", cnt::ops);
  cnt::ops = 0;
  const N se = nc::elem_sens<N>(xe, ve, gam, s, c);
  (void)se;
  std::printf("sens %lld\n", cnt::ops);
  cnt::ops = 0;
  nc::elem_linearize<N>(xe, gam, s, c, cache, 1);
  std::printf("linearize %lld\n", cnt::ops);
  cnt::ops = 0;
  nc::elem_jvp_lin<N>(cache, 1, ue, ve, gam, s, c, out);
  std::printf("jvp_lin %lld\n", cnt::ops);
  cnt::ops = 0;
  nc::elem_jtvp_lin<N>(cache, 1, ue, ve, gam, s, c, out);
  n = cnt::ops;
  std::printf("jtvp_lin %lld\n", n);
  return 0;
}
