// Arithmetic operation counts of the CUDA path's element routines, per element:
// the routines of nc_element.cuh instantiated with a number type that counts
// every +, -, * and / (one flop each, so an FMA counts 2) and every reciprocal
// square root (one flop), with unary minus free.  An operation between two
// compile-time constants (literals such as the Gauss-point weights and the
// products of them that the diagonal forms) is not counted: the compiler folds
// it.  Every value that reaches a routine at run time (nodal values, design,
// source, the kernel-wide constants of make_const) counts.  These are the
// algorithmic flop figures the benchmark's ALU roofline divides by the measured
// time.
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
// k: a compile-time constant (built from a literal); run-time values have k false
struct N {
  double v;
  bool k;
  N() : v(0.0), k(true) {}
  N(double x) : v(x), k(true) {}
  N(double x, bool konst) : v(x), k(konst) {}
};
inline N rt(double x) { return N(x, false); }
inline N op(double r, N a, N b) {
  if (!(a.k && b.k)) ++ops;
  return N(r, a.k && b.k);
}
inline N operator+(N a, N b) { return op(a.v + b.v, a, b); }
inline N operator-(N a, N b) { return op(a.v - b.v, a, b); }
inline N operator*(N a, N b) { return op(a.v * b.v, a, b); }
inline N operator/(N a, N b) { return op(a.v / b.v, a, b); }
inline N operator-(N a) { return N(-a.v, a.k); }
inline N& operator+=(N& a, N b) { a = a + b; return a; }
inline N& operator-=(N& a, N b) { a = a - b; return a; }
inline N& operator*=(N& a, N b) { a = a * b; return a; }
}  // namespace cnt

#include "../../paper_1508_04596_gb300/csrc/nc_element.cuh"

namespace nc {
template <>
inline cnt::N nc_rsqrt<cnt::N>(cnt::N v) {
  if (!v.k) ++cnt::ops;
  return cnt::N(1.0 / std::sqrt(v.v), v.k);
}
}  // namespace nc

using nc::ElemConst;
using cnt::N;

int main() {
  const double eg[3] = {0.0, 0.0, -1.0};
  ElemConst<N> c = nc::make_const<N>(1.0 / 64, 1e4, 0.71, 1e4, 1.0, 1.0, 0.1, eg);
  // the kernel-wide constants are kernel arguments: run-time values
  static_assert(sizeof(ElemConst<N>) % sizeof(N) == 0, "ElemConst holds N members only");
  N* cm = reinterpret_cast<N*>(&c);
  for (size_t i = 0; i < sizeof(ElemConst<N>) / sizeof(N); ++i) cm[i].k = false;
  N xe[5][8], ve[5][8], out[5][8], ue[3][8];
  for (int f = 0; f < 5; ++f)
    for (int a = 0; a < 8; ++a) {
      xe[f][a] = cnt::rt(0.1 * (f + 1) + 0.01 * a);
      ve[f][a] = cnt::rt(0.2 * (f + 1) - 0.03 * a);
    }
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 8; ++a) ue[i][a] = xe[i][a];
  const N gam = cnt::rt(0.4), s = cnt::rt(2.0);
  N cache[nc::LIN_SLOTS];  // written by elem_linearize from run-time values
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
