// Element-level arithmetic of the stabilised Q1-Q1 natural-convection residual.
//
// One trilinear hexahedron (edge h), 8 nodes x 5 unknowns (u, v, w, p, T), local
// node a = ia + 2 ja + 4 ka at reference corner (2ia-1, 2ja-1, 2ka-1).
// 2x2x2 Gauss quadrature (points +-1/sqrt(3), weight (h/2)^3).
//
// Physics (Sec. 2, Eq. 1a-c):  u.grad u - Pr div(grad u + grad u^T) + grad p
//   = -alpha u - Gr Pr^2 e^g T,  div u = 0,  u.grad T - div(K grad T) = s.
// Interpolation (Sec. 3.1, Eq. 7-8):  alpha(g) = amax (1-g)/(1+qa g),
//   K(g) = (g (Ck (1+qf) - 1) + 1) / (Ck (1 + qf g)).
// Stabilisation (App. B): tau = (tau1^-2 + tau2^-2 + tau3^-2)^-1/2 shared by SUPG
//   and PSPG, tau1 = 4h/||u_e||_2 (24 velocity unknowns), tau2 = h^2/(4 Pr),
//   tau3 = 1/alpha_e; thermal tau_T with h^2/(4 K_e) and no reaction limit.
// Weak form (the stabilised Galerkin form the paper cites, as read here):
//   r_{a,f} = sum_g w [ N_a f0_f + d_j N_a F1_{f,j} ],
//   f0_M = u.grad u + alpha u + beta e^g T,   F1_M[i][j] = Pr (G_ij + G_ji) - p d_ij + tau u_j rM_i
//   f0_C = div u,                             F1_C[j]    = tau rM_j
//   f0_T = rT,                                F1_T[j]    = K d_j T + tau_T u_j rT
//   rM_i = u.grad u_i + d_i p + alpha u_i + beta e^g_i T,  rT = u.grad T - s,  beta = Gr Pr^2.
//
// This header provides, for one element, the residual, its tangent (J v, with
// the dtau/du_e term of App. B), its adjoint (J^T w), the diagonal of J_e and
// the design derivative lambda^T dr_e/dgamma_e (with dtau/dgamma_e).  It is
// plain arithmetic on register arrays, usable from host and device code.
#pragma once
#include <cmath>

#if defined(__CUDACC__)
#define NC_HD __host__ __device__ __forceinline__
#else
#define NC_HD inline
#endif

namespace nc {

template <typename R>
struct ElemConst {
  R inv_h;      // 1/h
  R wq;         // Gauss weight (h/2)^3
  R Pr, beta;   // Pr, Gr Pr^2
  R eg[3];      // unit gravity direction
  R inv16h2;    // 1/(4h)^2      : tau1^-2 = S * inv16h2
  R t2inv2;     // (4 Pr/h^2)^2  : tau2^-2
  R k2c;        // (4/h^2)^2     : (h^2/(4K))^-2 = K^2 * k2c
  R amax, qa, qf, Ck;
};

template <typename R> NC_HD R nc_rsqrt(R v) {
#if defined(__CUDA_ARCH__)
  return rsqrt(v);
#else
  return R(1) / std::sqrt(v);
#endif
}

template <typename R> NC_HD R alpha_of(R g, const ElemConst<R>& c) {
  return c.amax * (R(1) - g) / (R(1) + c.qa * g);
}
template <typename R> NC_HD R dalpha_of(R g, const ElemConst<R>& c) {
  R d = R(1) + c.qa * g;
  return -c.amax * (R(1) + c.qa) / (d * d);
}
template <typename R> NC_HD R K_of(R g, const ElemConst<R>& c) {
  return (g * (c.Ck * (R(1) + c.qf) - R(1)) + R(1)) / (c.Ck * (R(1) + c.qf * g));
}
template <typename R> NC_HD R dK_of(R g, const ElemConst<R>& c) {
  R d = R(1) + c.qf * g;
  return ((c.Ck * (R(1) + c.qf) - R(1)) - c.qf) / (c.Ck * d * d);
}

// 1-D Q1 factors at the two Gauss points: node side i (0: -1, 1: +1), point side q.
NC_HD constexpr double gfac(int i, int q) {
  return i == q ? 0.78867513459481288225 : 0.21132486540518711775;  // (1 +- 1/sqrt 3)/2
}
NC_HD constexpr double gsgn(int i) { return i ? 1.0 : -1.0; }

// Value and physical gradient of one scalar nodal field at Gauss point (gx,gy,gz).
template <typename R, int gx, int gy, int gz>
NC_HD void interp(const R x[8], R inv_h, R& val, R grad[3]) {
  R v = R(0), dx = R(0), dy = R(0), dz = R(0);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int ia = a & 1, ja = (a >> 1) & 1, ka = (a >> 2) & 1;
    v += R(gfac(ia, gx) * gfac(ja, gy) * gfac(ka, gz)) * x[a];
    dx += R(gsgn(ia) * gfac(ja, gy) * gfac(ka, gz)) * x[a];
    dy += R(gfac(ia, gx) * gsgn(ja) * gfac(ka, gz)) * x[a];
    dz += R(gfac(ia, gx) * gfac(ja, gy) * gsgn(ka)) * x[a];
  }
  val = v;
  grad[0] = dx * inv_h;
  grad[1] = dy * inv_h;
  grad[2] = dz * inv_h;
}

// out[a] += N_a(g) f0 + d_j N_a(g) F1[j]   (F1 already carries 1/h)
template <typename R, int gx, int gy, int gz>
NC_HD void test_accum(R out[8], R f0, const R F1[3]) {
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int ia = a & 1, ja = (a >> 1) & 1, ka = (a >> 2) & 1;
    out[a] += R(gfac(ia, gx) * gfac(ja, gy) * gfac(ka, gz)) * f0 +
              R(gsgn(ia) * gfac(ja, gy) * gfac(ka, gz)) * F1[0] +
              R(gfac(ia, gx) * gsgn(ja) * gfac(ka, gz)) * F1[1] +
              R(gfac(ia, gx) * gfac(ja, gy) * gsgn(ka)) * F1[2];
  }
}

// Quadrature-point state: u, G[i][j] = d_j u_i, p, grad p, T, grad T.
template <typename R>
struct QP {
  R u[3], G[3][3], p, gp[3], T, gT[3];
};

template <typename R, int gx, int gy, int gz>
NC_HD void interp_all(const R xe[5][8], R inv_h, QP<R>& q) {
  interp<R, gx, gy, gz>(xe[0], inv_h, q.u[0], q.G[0]);
  interp<R, gx, gy, gz>(xe[1], inv_h, q.u[1], q.G[1]);
  interp<R, gx, gy, gz>(xe[2], inv_h, q.u[2], q.G[2]);
  interp<R, gx, gy, gz>(xe[3], inv_h, q.p, q.gp);
  interp<R, gx, gy, gz>(xe[4], inv_h, q.T, q.gT);
}

// Element coefficients shared by all Gauss points.
template <typename R>
struct ElemCoef {
  R alpha, K, tau, tauT, s;
};

template <typename R>
NC_HD ElemCoef<R> elem_coef(const R xe[5][8], R gam, R s, const ElemConst<R>& c, R& S) {
  ElemCoef<R> k;
  R acc = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) acc += xe[i][a] * xe[i][a];
  S = acc;
  k.alpha = alpha_of(gam, c);
  k.K = K_of(gam, c);
  k.tau = nc_rsqrt(S * c.inv16h2 + c.t2inv2 + k.alpha * k.alpha);
  k.tauT = nc_rsqrt(S * c.inv16h2 + k.K * k.K * c.k2c);
  k.s = s;
  return k;
}

// Strong residuals at a quadrature point.
template <typename R>
NC_HD void strong(const QP<R>& q, const ElemCoef<R>& k, const ElemConst<R>& c, R conv[3],
                  R rM[3], R& rT) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    conv[i] = q.u[0] * q.G[i][0] + q.u[1] * q.G[i][1] + q.u[2] * q.G[i][2];
    rM[i] = conv[i] + q.gp[i] + k.alpha * q.u[i] + c.beta * c.eg[i] * q.T;
  }
  rT = q.u[0] * q.gT[0] + q.u[1] * q.gT[1] + q.u[2] * q.gT[2] - k.s;
}

// ---------------------------------------------------------------------------- residual
template <typename R, int g>
NC_HD void gp_residual(const R xe[5][8], const ElemCoef<R>& k, const ElemConst<R>& c,
                       R out[5][8]) {
  constexpr int gx = g & 1, gy = (g >> 1) & 1, gz = (g >> 2) & 1;
  QP<R> q;
  interp_all<R, gx, gy, gz>(xe, c.inv_h, q);
  R conv[3], rM[3], rT;
  strong(q, k, c, conv, rM, rT);
  const R w = c.wq, wh = c.wq * c.inv_h;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R F1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
      F1[j] = wh * (c.Pr * (q.G[i][j] + q.G[j][i]) - (i == j ? q.p : R(0)) + k.tau * q.u[j] * rM[i]);
    test_accum<R, gx, gy, gz>(out[i], w * (conv[i] + k.alpha * q.u[i] + c.beta * c.eg[i] * q.T), F1);
  }
  {
    R F1[3] = {wh * k.tau * rM[0], wh * k.tau * rM[1], wh * k.tau * rM[2]};
    test_accum<R, gx, gy, gz>(out[3], w * (q.G[0][0] + q.G[1][1] + q.G[2][2]), F1);
  }
  {
    R F1[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) F1[j] = wh * (k.K * q.gT[j] + k.tauT * q.u[j] * rT);
    test_accum<R, gx, gy, gz>(out[4], w * rT, F1);
  }
}

template <typename R>
NC_HD void elem_residual(const R xe[5][8], R gam, R s, const ElemConst<R>& c, R out[5][8]) {
  R S;
  ElemCoef<R> k = elem_coef(xe, gam, s, c, S);
#pragma unroll
  for (int f = 0; f < 5; ++f)
#pragma unroll
    for (int a = 0; a < 8; ++a) out[f][a] = R(0);
  gp_residual<R, 0>(xe, k, c, out);
  gp_residual<R, 1>(xe, k, c, out);
  gp_residual<R, 2>(xe, k, c, out);
  gp_residual<R, 3>(xe, k, c, out);
  gp_residual<R, 4>(xe, k, c, out);
  gp_residual<R, 5>(xe, k, c, out);
  gp_residual<R, 6>(xe, k, c, out);
  gp_residual<R, 7>(xe, k, c, out);
}

// ---------------------------------------------------------------------------- tangent
// Directional derivative of the pointwise fluxes in the state direction dq and
// the parameter directions (dalpha, dK, dtau, dtauT); returns w-scaled f0 and
// (w/h)-scaled F1.
template <typename R>
NC_HD void flux_tangent(const QP<R>& q, const QP<R>& d, const ElemCoef<R>& k, R dalpha, R dK,
                        R dtau, R dtauT, const ElemConst<R>& c, R f0[5], R F1[5][3]) {
  R conv[3], rM[3], rT;
  strong(q, k, c, conv, rM, rT);
  R dconv[3], drM[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dconv[i] = d.u[0] * q.G[i][0] + d.u[1] * q.G[i][1] + d.u[2] * q.G[i][2] +
               q.u[0] * d.G[i][0] + q.u[1] * d.G[i][1] + q.u[2] * d.G[i][2];
    drM[i] = dconv[i] + d.gp[i] + k.alpha * d.u[i] + dalpha * q.u[i] + c.beta * c.eg[i] * d.T;
  }
  const R drT = d.u[0] * q.gT[0] + d.u[1] * q.gT[1] + d.u[2] * q.gT[2] +
                q.u[0] * d.gT[0] + q.u[1] * d.gT[1] + q.u[2] * d.gT[2];
  const R w = c.wq, wh = c.wq * c.inv_h;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    f0[i] = w * (dconv[i] + k.alpha * d.u[i] + dalpha * q.u[i] + c.beta * c.eg[i] * d.T);
#pragma unroll
    for (int j = 0; j < 3; ++j)
      F1[i][j] = wh * (c.Pr * (d.G[i][j] + d.G[j][i]) - (i == j ? d.p : R(0)) +
                       dtau * q.u[j] * rM[i] + k.tau * (d.u[j] * rM[i] + q.u[j] * drM[i]));
  }
  f0[3] = w * (d.G[0][0] + d.G[1][1] + d.G[2][2]);
#pragma unroll
  for (int j = 0; j < 3; ++j) F1[3][j] = wh * (dtau * rM[j] + k.tau * drM[j]);
  f0[4] = w * drT;
#pragma unroll
  for (int j = 0; j < 3; ++j)
    F1[4][j] = wh * (k.K * d.gT[j] + dK * q.gT[j] + dtauT * q.u[j] * rT +
                     k.tauT * (d.u[j] * rT + q.u[j] * drT));
}

template <typename R, int g>
NC_HD void gp_jvp(const R xe[5][8], const R ve[5][8], const ElemCoef<R>& k, R dtau, R dtauT,
                  const ElemConst<R>& c, R out[5][8]) {
  constexpr int gx = g & 1, gy = (g >> 1) & 1, gz = (g >> 2) & 1;
  QP<R> q, d;
  interp_all<R, gx, gy, gz>(xe, c.inv_h, q);
  interp_all<R, gx, gy, gz>(ve, c.inv_h, d);
  R f0[5], F1[5][3];
  flux_tangent(q, d, k, R(0), R(0), dtau, dtauT, c, f0, F1);
#pragma unroll
  for (int f = 0; f < 5; ++f) test_accum<R, gx, gy, gz>(out[f], f0[f], F1[f]);
}

// J_e v_e including the dtau/du_e and dtau_T/du_e terms (App. B).
template <typename R>
NC_HD void elem_jvp(const R xe[5][8], const R ve[5][8], R gam, R s, const ElemConst<R>& c,
                    R out[5][8]) {
  R S;
  ElemCoef<R> k = elem_coef(xe, gam, s, c, S);
  R uv = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) uv += xe[i][a] * ve[i][a];
  // d tau = -1/2 tau^3 d(S/(16h^2)),  dS = 2 u_e.v_e
  const R dtau = -k.tau * k.tau * k.tau * c.inv16h2 * uv;
  const R dtauT = -k.tauT * k.tauT * k.tauT * c.inv16h2 * uv;
#pragma unroll
  for (int f = 0; f < 5; ++f)
#pragma unroll
    for (int a = 0; a < 8; ++a) out[f][a] = R(0);
  gp_jvp<R, 0>(xe, ve, k, dtau, dtauT, c, out);
  gp_jvp<R, 1>(xe, ve, k, dtau, dtauT, c, out);
  gp_jvp<R, 2>(xe, ve, k, dtau, dtauT, c, out);
  gp_jvp<R, 3>(xe, ve, k, dtau, dtauT, c, out);
  gp_jvp<R, 4>(xe, ve, k, dtau, dtauT, c, out);
  gp_jvp<R, 5>(xe, ve, k, dtau, dtauT, c, out);
  gp_jvp<R, 6>(xe, ve, k, dtau, dtauT, c, out);
  gp_jvp<R, 7>(xe, ve, k, dtau, dtauT, c, out);
}

// ---------------------------------------------------------------------------- adjoint
// Given the interpolated test field w (value c0 and gradient C1 per field at the
// point), accumulate (dFlux/dq)^T (c0, C1) into the element output and return the
// cotangents of tau and tau_T.
template <typename R, int g>
NC_HD void gp_jtvp(const R xe[5][8], const R we[5][8], const ElemCoef<R>& k,
                   const ElemConst<R>& c, R out[5][8], R& tau_bar, R& tauT_bar) {
  constexpr int gx = g & 1, gy = (g >> 1) & 1, gz = (g >> 2) & 1;
  QP<R> q, t;
  interp_all<R, gx, gy, gz>(xe, c.inv_h, q);
  interp_all<R, gx, gy, gz>(we, c.inv_h, t);
  R conv[3], rM[3], rT;
  strong(q, k, c, conv, rM, rT);
  // cotangents of the fluxes: c0 = w * test value, C1 = w * test gradient
  const R w = c.wq;
  R c0[5] = {w * t.u[0], w * t.u[1], w * t.u[2], w * t.p, w * t.T};
  R C1[5][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    C1[0][j] = w * t.G[0][j];
    C1[1][j] = w * t.G[1][j];
    C1[2][j] = w * t.G[2][j];
    C1[3][j] = w * t.gp[j];
    C1[4][j] = w * t.gT[j];
  }
  R rMb[3], ub[3], Gb[3][3], gpb[3], gTb[3];
  const R C4u = C1[4][0] * q.u[0] + C1[4][1] * q.u[1] + C1[4][2] * q.u[2];
  const R rTb = c0[4] + k.tauT * C4u;
  R tb = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R Ciu = C1[i][0] * q.u[0] + C1[i][1] * q.u[1] + C1[i][2] * q.u[2];
    rMb[i] = k.tau * (Ciu + C1[3][i]);
    tb += Ciu * rM[i] + C1[3][i] * rM[i];
  }
  tau_bar += tb;
  tauT_bar += C4u * rT;
  R pb = -(C1[0][0] + C1[1][1] + C1[2][2]);
  R Tb = R(0);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    ub[j] = k.tau * (C1[0][j] * rM[0] + C1[1][j] * rM[1] + C1[2][j] * rM[2]) + k.tauT * C1[4][j] * rT;
    gTb[j] = k.K * C1[4][j] + rTb * q.u[j];
    gpb[j] = rMb[j];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Gb[i][j] = c.Pr * (C1[i][j] + C1[j][i]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R cb = c0[i] + rMb[i];  // cotangent of conv_i (and of the body terms)
    ub[i] += k.alpha * cb;
    Tb += c.beta * c.eg[i] * cb;
    Gb[i][i] += c0[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ub[j] += cb * q.G[i][j];
      Gb[i][j] += cb * q.u[j];
    }
  }
#pragma unroll
  for (int j = 0; j < 3; ++j) ub[j] += rTb * q.gT[j];
  const R ih = c.inv_h;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R F1[3] = {Gb[i][0] * ih, Gb[i][1] * ih, Gb[i][2] * ih};
    test_accum<R, gx, gy, gz>(out[i], ub[i], F1);
  }
  {
    R F1[3] = {gpb[0] * ih, gpb[1] * ih, gpb[2] * ih};
    test_accum<R, gx, gy, gz>(out[3], pb, F1);
  }
  {
    R F1[3] = {gTb[0] * ih, gTb[1] * ih, gTb[2] * ih};
    test_accum<R, gx, gy, gz>(out[4], Tb, F1);
  }
}

// J_e^T w_e.
template <typename R>
NC_HD void elem_jtvp(const R xe[5][8], const R we[5][8], R gam, R s, const ElemConst<R>& c,
                     R out[5][8]) {
  R S;
  ElemCoef<R> k = elem_coef(xe, gam, s, c, S);
#pragma unroll
  for (int f = 0; f < 5; ++f)
#pragma unroll
    for (int a = 0; a < 8; ++a) out[f][a] = R(0);
  R tb = R(0), tbT = R(0);
  gp_jtvp<R, 0>(xe, we, k, c, out, tb, tbT);
  gp_jtvp<R, 1>(xe, we, k, c, out, tb, tbT);
  gp_jtvp<R, 2>(xe, we, k, c, out, tb, tbT);
  gp_jtvp<R, 3>(xe, we, k, c, out, tb, tbT);
  gp_jtvp<R, 4>(xe, we, k, c, out, tb, tbT);
  gp_jtvp<R, 5>(xe, we, k, c, out, tb, tbT);
  gp_jtvp<R, 6>(xe, we, k, c, out, tb, tbT);
  gp_jtvp<R, 7>(xe, we, k, c, out, tb, tbT);
  // tau(S), S = u_e^T u_e:  d tau/d u_e = -tau^3/(16 h^2) u_e  (App. B)
  const R gsum = -(k.tau * k.tau * k.tau * tb + k.tauT * k.tauT * k.tauT * tbT) * c.inv16h2;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) out[i][a] += gsum * xe[i][a];
}

// ---------------------------------------------------------------------------- design derivative
template <typename R, int g>
NC_HD R gp_sens(const R xe[5][8], const R le[5][8], const ElemCoef<R>& k, R dalpha, R dK,
                R dtau, R dtauT, const ElemConst<R>& c) {
  constexpr int gx = g & 1, gy = (g >> 1) & 1, gz = (g >> 2) & 1;
  QP<R> q, t, zero;
  interp_all<R, gx, gy, gz>(xe, c.inv_h, q);
  interp_all<R, gx, gy, gz>(le, c.inv_h, t);
  zero.p = zero.T = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    zero.u[i] = zero.gp[i] = zero.gT[i] = R(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) zero.G[i][j] = R(0);
  }
  R f0[5], F1[5][3];
  flux_tangent(q, zero, k, dalpha, dK, dtau, dtauT, c, f0, F1);
  // F1 carries w/h; the test gradient below is the physical one times h
  const R h = R(1) / c.inv_h;
  R acc = f0[0] * t.u[0] + f0[1] * t.u[1] + f0[2] * t.u[2] + f0[3] * t.p + f0[4] * t.T;
#pragma unroll
  for (int j = 0; j < 3; ++j)
    acc += (F1[0][j] * t.G[0][j] + F1[1][j] * t.G[1][j] + F1[2][j] * t.G[2][j] +
            F1[3][j] * t.gp[j] + F1[4][j] * t.gT[j]) * h;
  return acc;
}

// lambda_e^T d r_e / d gamma_e, through alpha_e, K_e, tau(alpha_e), tau_T(K_e).
template <typename R>
NC_HD R elem_sens(const R xe[5][8], const R le[5][8], R gam, R s, const ElemConst<R>& c) {
  R S;
  ElemCoef<R> k = elem_coef(xe, gam, s, c, S);
  const R da = dalpha_of(gam, c), dK = dK_of(gam, c);
  // tau^-2 = S/(16h^2) + tau2^-2 + alpha^2  ->  dtau = -tau^3 alpha dalpha
  const R dtau = -k.tau * k.tau * k.tau * k.alpha * da;
  // tau_T^-2 = S/(16h^2) + K^2 (4/h^2)^2   ->  dtau_T = -tau_T^3 K k2c dK
  const R dtauT = -k.tauT * k.tauT * k.tauT * k.K * c.k2c * dK;
  R acc = R(0);
  acc += gp_sens<R, 0>(xe, le, k, da, dK, dtau, dtauT, c);
  acc += gp_sens<R, 1>(xe, le, k, da, dK, dtau, dtauT, c);
  acc += gp_sens<R, 2>(xe, le, k, da, dK, dtau, dtauT, c);
  acc += gp_sens<R, 3>(xe, le, k, da, dK, dtau, dtauT, c);
  acc += gp_sens<R, 4>(xe, le, k, da, dK, dtau, dtauT, c);
  acc += gp_sens<R, 5>(xe, le, k, da, dK, dtau, dtauT, c);
  acc += gp_sens<R, 6>(xe, le, k, da, dK, dtau, dtauT, c);
  acc += gp_sens<R, 7>(xe, le, k, da, dK, dtau, dtauT, c);
  return acc;
}

// ---------------------------------------------------------------------------- diagonal
// diag(J_e): the (a,f),(a,f) entries, from the diagonal blocks of the flux
// derivative (value slot and gradient slot of the same field) plus the tau
// coupling of the velocity rows.
template <typename R, int g>
NC_HD void gp_diag(const R xe[5][8], const ElemCoef<R>& k, const ElemConst<R>& c, R out[5][8],
                   R tcoup[3][8]) {
  constexpr int gx = g & 1, gy = (g >> 1) & 1, gz = (g >> 2) & 1;
  QP<R> q;
  interp_all<R, gx, gy, gz>(xe, c.inv_h, q);
  R conv[3], rM[3], rT;
  strong(q, k, c, conv, rM, rT);
  const R w = c.wq, ih = c.inv_h;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int ia = a & 1, ja = (a >> 1) & 1, ka = (a >> 2) & 1;
    const R N = R(gfac(ia, gx) * gfac(ja, gy) * gfac(ka, gz));
    const R D[3] = {R(gsgn(ia) * gfac(ja, gy) * gfac(ka, gz)) * ih,
                    R(gfac(ia, gx) * gsgn(ja) * gfac(ka, gz)) * ih,
                    R(gfac(ia, gx) * gfac(ja, gy) * gsgn(ka)) * ih};
    const R uD = q.u[0] * D[0] + q.u[1] * D[1] + q.u[2] * D[2];
    const R DD = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const R gi = q.G[i][i] + k.alpha;
      out[i][a] += w * (N * N * gi + N * uD + N * k.tau * (D[i] * rM[i] + uD * gi) +
                        c.Pr * (DD + D[i] * D[i]) + k.tau * uD * uD);
      tcoup[i][a] += w * uD * rM[i];
    }
    out[3][a] += w * k.tau * DD;
    out[4][a] += w * (N * uD + k.K * DD + k.tauT * uD * uD);
  }
}

template <typename R>
NC_HD void elem_diag(const R xe[5][8], R gam, R s, const ElemConst<R>& c, R out[5][8]) {
  R S;
  ElemCoef<R> k = elem_coef(xe, gam, s, c, S);
  R tc[3][8];
#pragma unroll
  for (int f = 0; f < 5; ++f)
#pragma unroll
    for (int a = 0; a < 8; ++a) out[f][a] = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) tc[i][a] = R(0);
  gp_diag<R, 0>(xe, k, c, out, tc);
  gp_diag<R, 1>(xe, k, c, out, tc);
  gp_diag<R, 2>(xe, k, c, out, tc);
  gp_diag<R, 3>(xe, k, c, out, tc);
  gp_diag<R, 4>(xe, k, c, out, tc);
  gp_diag<R, 5>(xe, k, c, out, tc);
  gp_diag<R, 6>(xe, k, c, out, tc);
  gp_diag<R, 7>(xe, k, c, out, tc);
  // d tau / d u_{a,i} = -tau^3/(16h^2) u_{a,i}
  const R dt = -k.tau * k.tau * k.tau * c.inv16h2;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) out[i][a] += dt * xe[i][a] * tc[i][a];
}

template <typename R>
NC_HD ElemConst<R> make_const(double h, double Gr, double Pr, double amax, double qa, double qf,
                              double Ck, const double eg[3]) {
  ElemConst<R> c;
  c.inv_h = R(1.0 / h);
  c.wq = R((h / 2) * (h / 2) * (h / 2));
  c.Pr = R(Pr);
  c.beta = R(Gr * Pr * Pr);
  c.eg[0] = R(eg[0]);
  c.eg[1] = R(eg[1]);
  c.eg[2] = R(eg[2]);
  c.inv16h2 = R(1.0 / (16.0 * h * h));
  c.t2inv2 = R((4.0 * Pr / (h * h)) * (4.0 * Pr / (h * h)));
  c.k2c = R((4.0 / (h * h)) * (4.0 / (h * h)));
  c.amax = R(amax);
  c.qa = R(qa);
  c.qf = R(qf);
  c.Ck = R(Ck);
  return c;
}

}  // namespace nc
