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
//
// Scaling.  Point gradients are kept in reference units, h grad (the nodal
// differences of the tensor-product stages, with no division by h), and so are
// the quantities formed from them: the strong residuals rM, rT and the value-slot
// fluxes f0 are h times their physical values.  The coefficients that meet them
// carry the compensating powers of h: alpha_e and the source s enter as h alpha,
// h s; tau, tau_T and K as tau/h, tau_T/h, K/h; the buoyancy vector as h beta e^g;
// the viscous weights as Pr wh/h; the value-slot Gauss weights as w/h.  The
// element rows come out in physical units.  This removes the 12 multiplications
// by 1/h per field and element that physical gradients would cost.
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
  R wh;         // wq / h: weight of the gradient-slot fluxes F1
  R wc[2];      // (wq/h) (1 -+ 1/sqrt 3)/2: the Gauss weight times the 1-D shape-function
                // weights of the (h-scaled) value-slot fluxes f0 (applied on the test side)
  R beg[3];     // h Gr Pr^2 e^g (buoyancy in the h-scaled strong residual)
  R prw, prw2;  // Pr wh/h, 2 Pr wh/h (viscous fluxes of reference gradients)
  R h;          // element edge
  R prh;        // Pr/h: the viscous cotangent weight on reference gradients
  R wdt;        // wh/16: weight of the tau derivative terms in scaled units
  R iwh;        // 1/wh: takes the store's SUPG weights wh tau rM back to tau rM
  R t2s;        // (4 Pr/h)^2 = h^2 tau2^-2: (tau/h)^-2 = S/16 + t2s + (h alpha)^2
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

// Along each axis a Q1 field at a Gauss point is a linear interpolation
// x0 + c (x1 - x0) with c = GW[q] (the shape-function weight of the "+" node), and
// the same difference (x1 - x0) is the derivative along that axis, so values and
// gradients share their differences (a tensor-product factorisation of the
// 2x2x2 rule).  Gradients are reference differences (h grad, see Scaling
// above).  interp_pair takes one pair of points
// (qy, qz fixed, qx = 0, 1); the diagonal of J uses it, every other element
// routine takes all 8 points at once (interp8 below).
constexpr double GW0 = 0.21132486540518711775;  // (1 - 1/sqrt 3)/2: weight of node 1 at point 0
constexpr double GW1 = 0.78867513459481288225;  // (1 + 1/sqrt 3)/2: weight of node 1 at point 1
NC_HD constexpr double gw(int q) { return q ? GW1 : GW0; }

template <typename R>
NC_HD void interp_pair(const R x[8], R cy, R cz, R val[2], R& gx, R gy[2], R gz[2]) {
  const R c0 = R(GW0), c1 = R(GW1);
  // z differences and interpolation at qz; index [ia][ja] <-> a = ia + 2 ja (+4 ka)
  const R dz00 = x[4] - x[0], dz10 = x[5] - x[1], dz01 = x[6] - x[2], dz11 = x[7] - x[3];
  const R z00 = x[0] + cz * dz00, z10 = x[1] + cz * dz10;
  const R z01 = x[2] + cz * dz01, z11 = x[3] + cz * dz11;
  // y differences and interpolation at qy, per ia
  const R dy0 = z01 - z00, dy1 = z11 - z10;
  const R y0 = z00 + cy * dy0, y1 = z10 + cy * dy1;
  // x
  const R dx = y1 - y0;
  val[0] = y0 + c0 * dx;
  val[1] = y0 + c1 * dx;
  gx = dx;
  const R ddy = dy1 - dy0;
  gy[0] = dy0 + c0 * ddy;
  gy[1] = dy0 + c1 * ddy;
  const R zy0 = dz00 + cy * (dz01 - dz00), zy1 = dz10 + cy * (dz11 - dz10);
  const R ddz = zy1 - zy0;
  gz[0] = zy0 + c0 * ddz;
  gz[1] = zy0 + c1 * ddz;
}

// Quadrature-point state: u, G[i][j] = d_j u_i, p, grad p, T, grad T.
template <typename R>
struct QP {
  R u[3], G[3][3], p, gp[3], T, gT[3];
};

template <typename R>
NC_HD void interp_field_pair(const R x[8], R cy, R cz, R v[2], R g[2][3]) {
  R val[2], gx, gy[2], gz[2];
  interp_pair<R>(x, cy, cz, val, gx, gy, gz);
  v[0] = val[0];
  v[1] = val[1];
  g[0][0] = gx;
  g[1][0] = gx;
  g[0][1] = gy[0];
  g[1][1] = gy[1];
  g[0][2] = gz[0];
  g[1][2] = gz[1];
}

template <typename R>
NC_HD void interp_all_pair(const R xe[5][8], R cy, R cz, QP<R> q[2]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R v[2], g[2][3];
    interp_field_pair<R>(xe[i], cy, cz, v, g);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      q[s].u[i] = v[s];
      q[s].G[i][0] = g[s][0];
      q[s].G[i][1] = g[s][1];
      q[s].G[i][2] = g[s][2];
    }
  }
  {
    R v[2], g[2][3];
    interp_field_pair<R>(xe[3], cy, cz, v, g);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      q[s].p = v[s];
      q[s].gp[0] = g[s][0];
      q[s].gp[1] = g[s][1];
      q[s].gp[2] = g[s][2];
    }
  }
  {
    R v[2], g[2][3];
    interp_field_pair<R>(xe[4], cy, cz, v, g);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      q[s].T = v[s];
      q[s].gT[0] = g[s][0];
      q[s].gT[1] = g[s][1];
      q[s].gT[2] = g[s][2];
    }
  }
}

// Element coefficients shared by all Gauss points, in the scaled units of the
// point quantities (see Scaling): alpha = h alpha_e, tau = tau_e/h,
// tau_T = tau_T,e/h, K = K_e/h, s = h s_e; wtau, wtauT, wK are tau, tau_T and K
// times the F1 weight wh.
template <typename R>
struct ElemCoef {
  R alpha, K, tau, tauT, s;
  R wtau, wtauT, wK;
};

template <typename R>
NC_HD void scale_coef(ElemCoef<R>& k, const ElemConst<R>& c) {
  k.wtau = c.wh * k.tau;
  k.wtauT = c.wh * k.tauT;
  k.wK = c.wh * k.K;
}

template <typename R>
NC_HD ElemCoef<R> elem_coef(const R xe[5][8], R gam, R s, const ElemConst<R>& c, R& S) {
  ElemCoef<R> k;
  R acc = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) acc += xe[i][a] * xe[i][a];
  S = acc;
  k.alpha = c.h * alpha_of(gam, c);
  k.K = c.inv_h * K_of(gam, c);
  // (tau_e/h)^-2 = h^2 (S/(4h)^2 + (4 Pr/h^2)^2 + alpha_e^2) and
  // (tau_T,e/h)^-2 = h^2 (S/(4h)^2 + (4 K_e/h^2)^2) in the scaled coefficients
  k.tau = nc_rsqrt(S * R(0.0625) + c.t2s + k.alpha * k.alpha);
  k.tauT = nc_rsqrt(S * R(0.0625) + k.K * k.K * R(16));
  k.s = c.h * s;
  scale_coef(k, c);
  return k;
}

// Strong residuals at a quadrature point; body = rM without the pressure
// gradient (convection, Brinkman friction and buoyancy), the value-slot flux of
// the momentum rows.
template <typename R>
NC_HD void strong(const QP<R>& q, const ElemCoef<R>& k, const ElemConst<R>& c, R body[3],
                  R rM[3], R& rT) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    body[i] = q.u[0] * q.G[i][0] + q.u[1] * q.G[i][1] + q.u[2] * q.G[i][2] + k.alpha * q.u[i] +
              c.beg[i] * q.T;
    rM[i] = body[i] + q.gp[i];
  }
  rT = q.u[0] * q.gT[0] + q.u[1] * q.gT[1] + q.u[2] * q.gT[2] - k.s;
}

// Gradient-slot momentum fluxes shared by the residual and its tangent:
// F1[i][j] = Pr wh (G_ij + G_ji) - delta_ij pw + u_j a_i (+ v_j b_i with HASV; the
// viscous part formed once per symmetric pair).
template <typename R, bool HASV>
NC_HD void momentum_F1(const R G[3][3], R pw, const R u[3], const R a[3], const R v[3],
                       const R b[3], const ElemConst<R>& c, R F1[5][3]) {
  const R v01 = c.prw * (G[0][1] + G[1][0]);
  const R v02 = c.prw * (G[0][2] + G[2][0]);
  const R v12 = c.prw * (G[1][2] + G[2][1]);
  const R vd[3] = {c.prw2 * G[0][0] - pw, c.prw2 * G[1][1] - pw, c.prw2 * G[2][2] - pw};
  const R vo[3][3] = {{vd[0], v01, v02}, {v01, vd[1], v12}, {v02, v12, vd[2]}};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      F1[i][j] = HASV ? vo[i][j] + u[j] * a[i] + v[j] * b[i] : vo[i][j] + u[j] * a[i];
}

// ---------------------------------------------------------------------------- residual
// Pointwise fluxes of the residual: f0 (the Gauss weight is applied on the test
// side) and (w/h)-scaled F1.
template <typename R>
NC_HD void flux_residual(const QP<R>& q, const ElemCoef<R>& k, const ElemConst<R>& c, R f0[5],
                         R F1[5][3]) {
  R body[3], rM[3], rT;
  strong(q, k, c, body, rM, rT);
  R b[3];  // wh tau rM: the SUPG weight of the momentum rows and the PSPG flux
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    b[i] = k.wtau * rM[i];
    f0[i] = body[i];
    F1[3][i] = b[i];
  }
  momentum_F1<R, false>(q.G, c.wh * q.p, q.u, b, q.u, b, c, F1);
  f0[3] = q.G[0][0] + q.G[1][1] + q.G[2][2];
  f0[4] = rT;
  const R trT = k.wtauT * rT;
#pragma unroll
  for (int j = 0; j < 3; ++j) F1[4][j] = k.wK * q.gT[j] + q.u[j] * trT;
}

template <typename R>
NC_HD void zero_out(R out[5][8]) {
#pragma unroll
  for (int f = 0; f < 5; ++f)
#pragma unroll
    for (int a = 0; a < 8; ++a) out[f][a] = R(0);
}

// ---------------------------------------------------------------------------- tangent
// Directional derivative of the pointwise fluxes in the state direction d and,
// with PARAM, the parameter directions (dalpha, dK); dtau, dtauT are the
// derivatives of tau, tau_T along the same direction.  Returns f0 (the Gauss
// weight is applied on the test side) and (w/h)-scaled F1.  Without PARAM,
// dalpha and dK are not read (J v needs none).  With STORE (the products from
// the linearisation store), rM and rT hold the SUPG weights wtau rM, wtauT rT
// of the store, and dtau, dtauT the ratios dtau/tau, dtauT/tauT: the terms
// dtau rM then cost one multiplication each, and the weights none.
template <typename R, bool PARAM, bool STORE = false>
NC_HD void flux_tangent_rm(const QP<R>& q, const R rM[3], R rT, const QP<R>& d,
                           const ElemCoef<R>& k, R dalpha, R dK, R dtau, R dtauT,
                           const ElemConst<R>& c, R f0[5], R F1[5][3]) {
  const R whdtau = STORE ? dtau : c.wh * dtau;
  R a[3], b[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    // derivative of rM_i without the pressure gradient (the value-slot flux)
    R body = d.u[0] * q.G[i][0] + d.u[1] * q.G[i][1] + d.u[2] * q.G[i][2] + q.u[0] * d.G[i][0] +
             q.u[1] * d.G[i][1] + q.u[2] * d.G[i][2] + k.alpha * d.u[i] + c.beg[i] * d.T;
    if (PARAM) body += dalpha * q.u[i];
    const R drM = body + d.gp[i];
    f0[i] = body;
    // d(tau u_j rM_i) = u_j (dtau rM_i + tau drM_i) + d.u_j (tau rM_i), times wh
    a[i] = whdtau * rM[i] + k.wtau * drM;
    b[i] = STORE ? rM[i] : k.wtau * rM[i];
    F1[3][i] = a[i];
  }
  momentum_F1<R, true>(d.G, c.wh * d.p, q.u, a, d.u, b, c, F1);
  const R drT = d.u[0] * q.gT[0] + d.u[1] * q.gT[1] + d.u[2] * q.gT[2] + q.u[0] * d.gT[0] +
                q.u[1] * d.gT[1] + q.u[2] * d.gT[2];
  f0[3] = d.G[0][0] + d.G[1][1] + d.G[2][2];
  f0[4] = drT;
  const R aT = (STORE ? dtauT : c.wh * dtauT) * rT + k.wtauT * drT;
  const R bT = STORE ? rT : k.wtauT * rT;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    R t = k.wK * d.gT[j] + q.u[j] * aT + d.u[j] * bT;
    if (PARAM) t += (c.wh * dK) * q.gT[j];
    F1[4][j] = t;
  }
}

template <typename R, bool PARAM>
NC_HD void flux_tangent(const QP<R>& q, const QP<R>& d, const ElemCoef<R>& k, R dalpha, R dK,
                        R dtau, R dtauT, const ElemConst<R>& c, R f0[5], R F1[5][3]) {
  R body[3], rM[3], rT;
  strong(q, k, c, body, rM, rT);
  flux_tangent_rm<R, PARAM>(q, rM, rT, d, k, dalpha, dK, dtau, dtauT, c, f0, F1);
}

// ---------------------------------------------------------------------------- adjoint
// Given the interpolated test field t (value and gradient per field at the
// point), the cotangents of the point state, (dFlux/dq)^T (w t), returned as
// f0 (value slots, without the Gauss weight, which the test side applies) and F1
// (gradient slots, times w/h) for the test-side transpose, plus the cotangents
// of tau and tau_T accumulated WITHOUT the Gauss weight w (the caller applies it
// once per element).  The weight is applied to the outputs rather than to the 20
// seeds, and the symmetric viscous cotangent is formed once per pair (i, j).
// With STORE, rM and rT hold the store's SUPG weights wtau rM, wtauT rT; the
// cotangents of tau and tau_T then come out multiplied by wh tau and wh tau_T
// (the caller divides them out once per element).
template <typename R, bool STORE = false>
NC_HD void flux_adjoint_rm(const QP<R>& q, const R rM[3], R rT, const QP<R>& t,
                           const ElemCoef<R>& k, const ElemConst<R>& c, R f0[5], R F1[5][3],
                           R& tau_bar, R& tauT_bar) {
  // seeds: c0 = test values, C1 = test gradients (unweighted)
  const R* const C1[5] = {t.G[0], t.G[1], t.G[2], t.gp, t.gT};
  const R c0[5] = {t.u[0], t.u[1], t.u[2], t.p, t.T};
  R rMb[3], ub[3], Gb[3][3], gTb[3];
  const R C4u = C1[4][0] * q.u[0] + C1[4][1] * q.u[1] + C1[4][2] * q.u[2];
  const R rTb = c0[4] + k.tauT * C4u;
  R tb = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R s = C1[i][0] * q.u[0] + C1[i][1] * q.u[1] + C1[i][2] * q.u[2] + C1[3][i];
    rMb[i] = k.tau * s;
    tb += s * rM[i];
  }
  tau_bar += tb;
  tauT_bar += C4u * rT;
  const R pb = -(C1[0][0] + C1[1][1] + C1[2][2]);
  R Tb = R(0);
  const R trT = (STORE ? c.iwh : k.tauT) * rT;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    ub[j] = (STORE ? c.iwh : k.tau) * (C1[0][j] * rM[0] + C1[1][j] * rM[1] + C1[2][j] * rM[2]) +
            C1[4][j] * trT + rTb * q.gT[j];
    gTb[j] = k.K * C1[4][j] + rTb * q.u[j];
  }
  {
    const R g01 = c.prh * (C1[0][1] + C1[1][0]), g02 = c.prh * (C1[0][2] + C1[2][0]);
    const R g12 = c.prh * (C1[1][2] + C1[2][1]);
    const R p2 = R(2) * c.prh;
    Gb[0][0] = p2 * C1[0][0] + c0[3];
    Gb[1][1] = p2 * C1[1][1] + c0[3];
    Gb[2][2] = p2 * C1[2][2] + c0[3];
    Gb[0][1] = Gb[1][0] = g01;
    Gb[0][2] = Gb[2][0] = g02;
    Gb[1][2] = Gb[2][1] = g12;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R cb = c0[i] + rMb[i];  // cotangent of conv_i (and of the body terms)
    ub[i] += k.alpha * cb;
    Tb += c.beg[i] * cb;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ub[j] += cb * q.G[i][j];
      Gb[i][j] += cb * q.u[j];
    }
  }
  const R wh = c.wh;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    f0[i] = ub[i];
    F1[i][0] = wh * Gb[i][0];
    F1[i][1] = wh * Gb[i][1];
    F1[i][2] = wh * Gb[i][2];
    F1[3][i] = wh * rMb[i];
    F1[4][i] = wh * gTb[i];
  }
  f0[3] = pb;
  f0[4] = Tb;
}

template <typename R>
NC_HD void flux_adjoint(const QP<R>& q, const QP<R>& t, const ElemCoef<R>& k,
                        const ElemConst<R>& c, R f0[5], R F1[5][3], R& tau_bar, R& tauT_bar) {
  R conv[3], rM[3], rT;
  strong(q, k, c, conv, rM, rT);
  flux_adjoint_rm(q, rM, rT, t, k, c, f0, F1, tau_bar, tauT_bar);
}

// ---------------------------------------------------------------------------- design derivative
// lambda^T dr/dgamma at one Gauss point: the tangent fluxes of flux_tangent_rm
// in the parameter directions alone (the state direction is zero), contracted
// with the test field t.  With no state direction only these terms remain:
//   f0_M[i] = dalpha u_i,   F1_M[i][j] = u_j a_i,   F1_C[i] = a_i,
//   a_i = wh (dtau rM_i + tau dalpha u_i),
//   F1_T[j] = u_j wh dtauT rT + wh dK grad_j T,
// so the contraction is  wh sum_i f0_M[i] t.u_i
//   + sum_i a_i (u . grad t_i + d_i t_p) + wh dtauT rT (u . grad t_T)
//   + wh dK (grad T . grad t_T)
// (f0 is h-scaled and takes the weight w/h; F1 carries w/h and meets the test
// gradients in reference units, which supply the missing h).
template <typename R>
NC_HD R point_sens(const QP<R>& q, const QP<R>& t, const ElemCoef<R>& k, R dalpha, R dK, R dtau,
                   R dtauT, const ElemConst<R>& c) {
  R body[3], rM[3], rT;
  strong(q, k, c, body, rM, rT);
  const R whdtau = c.wh * dtau;
  R acc = R(0), acc1 = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const R f0 = dalpha * q.u[i];
    acc += f0 * t.u[i];
    const R a = whdtau * rM[i] + k.wtau * f0;
    acc1 += a * (q.u[0] * t.G[i][0] + q.u[1] * t.G[i][1] + q.u[2] * t.G[i][2] + t.gp[i]);
  }
  const R ugT = q.u[0] * t.gT[0] + q.u[1] * t.gT[1] + q.u[2] * t.gT[2];
  const R gTgT = q.gT[0] * t.gT[0] + q.gT[1] * t.gT[1] + q.gT[2] * t.gT[2];
  acc1 += (c.wh * dtauT) * rT * ugT + (c.wh * dK) * gTgT;
  return c.wh * acc + acc1;
}

// ---------------------------------------------------------------------------- linearisation cache
// In a Krylov solve J is applied many times at one state.  The state-only part
// of every Gauss point -- u, grad u, grad T and the strong residuals rM, rT --
// and the element's tau, tau_T can be computed once per linearisation and read
// back by each product instead of being re-interpolated.  Layout: point g' =
// 2 * pair + qx (pairs in the order (qy, qz) = (0,0), (1,0), (0,1), (1,1)),
// LIN_GP values per point (u[3], G[3][3], gT[3], and the SUPG weights of the
// strong residuals, wtau rM[3] and wtauT rT, which the products use as they
// are), then tau, tau_T,
// alpha, K (all in the scaled units of the point quantities, see Scaling; alpha
// and K are stored so that the products need no division);
// slot s of an element is stored at cache[s * stride].
constexpr int LIN_GP = 19;
constexpr int LIN_SLOTS = 8 * LIN_GP + 4;

template <typename R>
NC_HD void load_lin_pair(const R* cache, long long stride, int P, QP<R> q[2], R rM[2][3], R rT[2]) {
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const R* o = cache + (long long)((2 * P + s) * LIN_GP) * stride;
#pragma unroll
    for (int i = 0; i < 3; ++i) q[s].u[i] = o[i * stride];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) q[s].G[i][j] = o[(3 + 3 * i + j) * stride];
#pragma unroll
    for (int j = 0; j < 3; ++j) q[s].gT[j] = o[(12 + j) * stride];
#pragma unroll
    for (int i = 0; i < 3; ++i) rM[s][i] = o[(15 + i) * stride];
    rT[s] = o[18 * stride];
    q[s].p = q[s].T = R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) q[s].gp[i] = R(0);
  }
}

template <typename R>
NC_HD ElemCoef<R> lin_coef(const R* cache, long long stride, R gam, R s, const ElemConst<R>& c) {
  (void)gam;  // alpha and K come from the store
  ElemCoef<R> k;
  k.tau = cache[(long long)(8 * LIN_GP) * stride];
  k.tauT = cache[(long long)(8 * LIN_GP + 1) * stride];
  k.alpha = cache[(long long)(8 * LIN_GP + 2) * stride];
  k.K = cache[(long long)(8 * LIN_GP + 3) * stride];
  k.s = c.h * s;
  scale_coef(k, c);
  return k;
}

// ---------------------------------------------------------------------------- diagonal
// diag(J_e): the (a,f),(a,f) entries, from the diagonal blocks of the flux
// derivative (value slot and gradient slot of the same field) plus the tau
// coupling of the velocity rows.
template <typename R, int gx, int gy, int gz>
NC_HD void point_diag(const QP<R>& q, const ElemCoef<R>& k, const ElemConst<R>& c, R out[5][8],
                      R tcoup[3][8]) {
  R conv[3], rM[3], rT;
  strong(q, k, c, conv, rM, rT);
  const R w = c.wh;  // the weight w/h: every term below is h times its physical value
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int ia = a & 1, ja = (a >> 1) & 1, ka = (a >> 2) & 1;
    const R N = R(gfac(ia, gx) * gfac(ja, gy) * gfac(ka, gz));
    const R D[3] = {R(gsgn(ia) * gfac(ja, gy) * gfac(ka, gz)),
                    R(gfac(ia, gx) * gsgn(ja) * gfac(ka, gz)),
                    R(gfac(ia, gx) * gfac(ja, gy) * gsgn(ka))};
    const R uD = q.u[0] * D[0] + q.u[1] * D[1] + q.u[2] * D[2];
    const R DD = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const R gi = q.G[i][i] + k.alpha;
      out[i][a] += w * (N * N * gi + N * uD + N * k.tau * (D[i] * rM[i] + uD * gi) +
                        c.prh * (DD + D[i] * D[i]) + k.tau * uD * uD);
      tcoup[i][a] += w * uD * rM[i];
    }
    out[3][a] += w * k.tau * DD;
    out[4][a] += w * (N * uD + k.K * DD + k.tauT * uD * uD);
  }
}

template <typename R, int qy, int qz>
NC_HD void pair_diag(const R xe[5][8], const ElemCoef<R>& k, const ElemConst<R>& c, R out[5][8],
                     R tcoup[3][8]) {
  QP<R> q[2];
  interp_all_pair<R>(xe, R(gw(qy)), R(gw(qz)), q);
  point_diag<R, 0, qy, qz>(q[0], k, c, out, tcoup);
  point_diag<R, 1, qy, qz>(q[1], k, c, out, tcoup);
}

template <typename R>
NC_HD void elem_diag(const R xe[5][8], R gam, R s, const ElemConst<R>& c, R out[5][8]) {
  R S;
  ElemCoef<R> k = elem_coef(xe, gam, s, c, S);
  R tc[3][8];
  zero_out(out);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) tc[i][a] = R(0);
  pair_diag<R, 0, 0>(xe, k, c, out, tc);
  pair_diag<R, 1, 0>(xe, k, c, out, tc);
  pair_diag<R, 0, 1>(xe, k, c, out, tc);
  pair_diag<R, 1, 1>(xe, k, c, out, tc);
  // d tau_e / d u_{a,i} = -tau_e^3/(16h^2) u_{a,i}; in the scaled units of tc
  // (h^2 times physical, the weight w/h) and of tau this is -tau^3/16
  const R dt = -k.tau * k.tau * k.tau * R(0.0625);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) out[i][a] += dt * xe[i][a] * tc[i][a];
}

// ---------------------------------------------------------------------------- element routines
// The tensor-product factorisation is taken over the whole element: per field,
// the z stage (column differences and values at both qz), the y stage
// (differences and values at both qy, and the z-difference interpolated in y)
// and the x stage are each formed once for all 8 points (102 flop per field;
// 176 when the points are taken pair by pair), and the test side is their exact
// transpose (134 flop; 196 pair by pair).  Point index p = qx + 2 qy + 4 qz (the
// order of the linearisation store).  All 8 points are live at once: more
// local-memory traffic, fewer instructions, which measured faster in both
// precisions.
NC_HD constexpr int pt(int qx, int qy, int qz) { return qx + 2 * qy + 4 * qz; }

// Values and (1/h-scaled) gradients of one Q1 field at the 8 Gauss points.
template <typename R>
NC_HD void interp8(const R x[8], R val[8], R g[8][3]) {
  const R c[2] = {R(GW0), R(GW1)};
  R dz[4], vz[2][4];
#pragma unroll
  for (int col = 0; col < 4; ++col) {  // column col = ia + 2 ja: nodes col, col + 4
    dz[col] = x[col + 4] - x[col];
    vz[0][col] = x[col] + c[0] * dz[col];
    vz[1][col] = x[col] + c[1] * dz[col];
  }
  R dy[2][2], vyz[2][2][2];  // [qz][ia], [qz][qy][ia]
#pragma unroll
  for (int qz = 0; qz < 2; ++qz)
#pragma unroll
    for (int ia = 0; ia < 2; ++ia) {
      dy[qz][ia] = vz[qz][ia + 2] - vz[qz][ia];
      vyz[qz][0][ia] = vz[qz][ia] + c[0] * dy[qz][ia];
      vyz[qz][1][ia] = vz[qz][ia] + c[1] * dy[qz][ia];
    }
  R dzy[2][2];  // z-difference interpolated in y: [qy][ia]
#pragma unroll
  for (int ia = 0; ia < 2; ++ia) {
    const R ez = dz[ia + 2] - dz[ia];
    dzy[0][ia] = dz[ia] + c[0] * ez;
    dzy[1][ia] = dz[ia] + c[1] * ez;
  }
#pragma unroll
  for (int qz = 0; qz < 2; ++qz)
#pragma unroll
    for (int qy = 0; qy < 2; ++qy) {
      const R dx = vyz[qz][qy][1] - vyz[qz][qy][0];
      const R gxv = dx;
#pragma unroll
      for (int qx = 0; qx < 2; ++qx) {
        val[pt(qx, qy, qz)] = vyz[qz][qy][0] + c[qx] * dx;
        g[pt(qx, qy, qz)][0] = gxv;
      }
    }
#pragma unroll
  for (int qz = 0; qz < 2; ++qz) {
    const R ey = dy[qz][1] - dy[qz][0];
#pragma unroll
    for (int qx = 0; qx < 2; ++qx) {
      const R gyv = dy[qz][0] + c[qx] * ey;
      g[pt(qx, 0, qz)][1] = gyv;
      g[pt(qx, 1, qz)][1] = gyv;
    }
  }
#pragma unroll
  for (int qy = 0; qy < 2; ++qy) {
    const R ex = dzy[qy][1] - dzy[qy][0];
#pragma unroll
    for (int qx = 0; qx < 2; ++qx) {
      const R gzv = dzy[qy][0] + c[qx] * ex;
      g[pt(qx, qy, 0)][2] = gzv;
      g[pt(qx, qy, 1)][2] = gzv;
    }
  }
}

// Transpose of interp8 (without the 1/h, which the caller folds into F1):
// out[a] = sum_p [ w N_a(p) f0[p] + dN_a/dxi_j(p) F1[p][j] ] (written, not added:
// a sum onto zeros would cost an addition per row), with the Gauss
// weight of the (h-scaled) value slots applied here: wc = (w/h) (1 -+ 1/sqrt 3)/2.  The x stage
// takes the two points of a pair to the two nodes: node 1 gets
// wc0 f0[p0] + wc1 f0[p1] + F, node 0 gets wc1 f0[p0] + wc0 f0[p1] - F (the 1-D
// weights of node 0 are those of node 1 mirrored), F the pair's x-gradient fluxes.
template <typename R>
NC_HD void test8(R out[8], const R f0[8], const R F1[8][3], const R wc[2]) {
  const R c[2] = {R(GW0), R(GW1)};
  R vyzb[2][2][2], dyb[2][2], dzyb[2][2];
#pragma unroll
  for (int qz = 0; qz < 2; ++qz)
#pragma unroll
    for (int qy = 0; qy < 2; ++qy) {
      const int p0 = pt(0, qy, qz), p1 = pt(1, qy, qz);
      const R F = F1[p0][0] + F1[p1][0];
      vyzb[qz][qy][1] = wc[0] * f0[p0] + (wc[1] * f0[p1] + F);
      vyzb[qz][qy][0] = wc[1] * f0[p0] + (wc[0] * f0[p1] - F);
    }
#pragma unroll
  for (int qz = 0; qz < 2; ++qz) {
    const R b0 = F1[pt(0, 0, qz)][1] + F1[pt(0, 1, qz)][1];
    const R b1 = F1[pt(1, 0, qz)][1] + F1[pt(1, 1, qz)][1];
    const R eyb = c[0] * b0 + c[1] * b1;
    dyb[qz][0] = b0 + b1 - eyb;
    dyb[qz][1] = eyb;
  }
#pragma unroll
  for (int qy = 0; qy < 2; ++qy) {
    const R b0 = F1[pt(0, qy, 0)][2] + F1[pt(0, qy, 1)][2];
    const R b1 = F1[pt(1, qy, 0)][2] + F1[pt(1, qy, 1)][2];
    const R exb = c[0] * b0 + c[1] * b1;
    dzyb[qy][0] = b0 + b1 - exb;
    dzyb[qy][1] = exb;
  }
  R vzb[2][4];
#pragma unroll
  for (int qz = 0; qz < 2; ++qz)
#pragma unroll
    for (int ia = 0; ia < 2; ++ia) {
      const R d = dyb[qz][ia] + c[0] * vyzb[qz][0][ia] + c[1] * vyzb[qz][1][ia];
      vzb[qz][ia] = vyzb[qz][0][ia] + vyzb[qz][1][ia] - d;
      vzb[qz][ia + 2] = d;
    }
  R dzb[4];
#pragma unroll
  for (int ia = 0; ia < 2; ++ia) {
    const R ezb = c[0] * dzyb[0][ia] + c[1] * dzyb[1][ia];
    dzb[ia] = dzyb[0][ia] + dzyb[1][ia] - ezb;
    dzb[ia + 2] = ezb;
  }
#pragma unroll
  for (int col = 0; col < 4; ++col) {
    const R d = dzb[col] + c[0] * vzb[0][col] + c[1] * vzb[1][col];
    out[col] = vzb[0][col] + vzb[1][col] - d;
    out[col + 4] = d;
  }
}

template <typename R>
NC_HD void interp_all8(const R xe[5][8], QP<R> q[8]) {
  R val[8], g[8][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    interp8<R>(xe[i], val, g);
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      q[p].u[i] = val[p];
      q[p].G[i][0] = g[p][0];
      q[p].G[i][1] = g[p][1];
      q[p].G[i][2] = g[p][2];
    }
  }
  interp8<R>(xe[3], val, g);
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    q[p].p = val[p];
    q[p].gp[0] = g[p][0];
    q[p].gp[1] = g[p][1];
    q[p].gp[2] = g[p][2];
  }
  interp8<R>(xe[4], val, g);
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    q[p].T = val[p];
    q[p].gT[0] = g[p][0];
    q[p].gT[1] = g[p][1];
    q[p].gT[2] = g[p][2];
  }
}

template <typename R>
NC_HD void test_all8(R out[5][8], const R f0[8][5], const R F1[8][5][3], const R wc[2]) {
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    R a[8], b[8][3];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      a[p] = f0[p][f];
      b[p][0] = F1[p][f][0];
      b[p][1] = F1[p][f][1];
      b[p][2] = F1[p][f][2];
    }
    test8<R>(out[f], a, b, wc);
  }
}

template <typename R>
NC_HD void elem_residual(const R xe[5][8], R gam, R s, const ElemConst<R>& c, R out[5][8]) {
  R S;
  const ElemCoef<R> k = elem_coef(xe, gam, s, c, S);
  QP<R> q[8];
  interp_all8<R>(xe, q);
  R f0[8][5], F1[8][5][3];
#pragma unroll
  for (int p = 0; p < 8; ++p) flux_residual(q[p], k, c, f0[p], F1[p]);
  test_all8<R>(out, f0, F1, c.wc);
}

template <typename R>
NC_HD void elem_jvp(const R xe[5][8], const R ve[5][8], R gam, R s, const ElemConst<R>& c,
                     R out[5][8]) {
  R S;
  const ElemCoef<R> k = elem_coef(xe, gam, s, c, S);
  R uv = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) uv += xe[i][a] * ve[i][a];
  // d tau_e = -tau_e^3 uv/(16 h^2); scaled (d tau_e / h): -tau^3 uv/16
  const R dtau = -k.tau * k.tau * k.tau * R(0.0625) * uv;
  const R dtauT = -k.tauT * k.tauT * k.tauT * R(0.0625) * uv;
  QP<R> q[8], d[8];
  interp_all8<R>(xe, q);
  interp_all8<R>(ve, d);
  R f0[8][5], F1[8][5][3];
#pragma unroll
  for (int p = 0; p < 8; ++p)
    flux_tangent<R, false>(q[p], d[p], k, R(0), R(0), dtau, dtauT, c, f0[p], F1[p]);
  test_all8<R>(out, f0, F1, c.wc);
}

template <typename R>
NC_HD void elem_jtvp(const R xe[5][8], const R we[5][8], R gam, R s, const ElemConst<R>& c,
                      R out[5][8]) {
  R S;
  const ElemCoef<R> k = elem_coef(xe, gam, s, c, S);
  QP<R> q[8], t[8];
  interp_all8<R>(xe, q);
  interp_all8<R>(we, t);
  R f0[8][5], F1[8][5][3];
  R tb = R(0), tbT = R(0);
#pragma unroll
  for (int p = 0; p < 8; ++p) flux_adjoint(q[p], t[p], k, c, f0[p], F1[p], tb, tbT);
  test_all8<R>(out, f0, F1, c.wc);
  const R gsum = -(k.tau * k.tau * k.tau * tb + k.tauT * k.tauT * k.tauT * tbT) * c.wdt;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) out[i][a] += gsum * xe[i][a];
}

template <typename R>
NC_HD R elem_sens(const R xe[5][8], const R le[5][8], R gam, R s, const ElemConst<R>& c) {
  R S;
  const ElemCoef<R> k = elem_coef(xe, gam, s, c, S);
  // design derivatives in the scaled units of the coefficients: d(h alpha_e),
  // d(K_e/h), and of tau, tau_T from (tau)^-2 = S/16 + t2s + alpha^2 and
  // (tau_T)^-2 = S/16 + 16 K^2
  const R da = c.h * dalpha_of(gam, c), dK = c.inv_h * dK_of(gam, c);
  const R dtau = -k.tau * k.tau * k.tau * k.alpha * da;
  const R dtauT = -k.tauT * k.tauT * k.tauT * k.K * R(16) * dK;
  QP<R> q[8], t[8];
  interp_all8<R>(xe, q);
  interp_all8<R>(le, t);
  R acc = R(0);
#pragma unroll
  for (int p = 0; p < 8; ++p) acc += point_sens(q[p], t[p], k, da, dK, dtau, dtauT, c);
  return acc;
}

template <typename R>
NC_HD void elem_linearize(const R xe[5][8], R gam, R s, const ElemConst<R>& c, R* cache,
                           long long stride) {
  R S;
  const ElemCoef<R> k = elem_coef(xe, gam, s, c, S);
  QP<R> q[8];
  interp_all8<R>(xe, q);
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    R body[3], rM[3], rT;
    strong(q[p], k, c, body, rM, rT);
    R* o = cache + (long long)(p * LIN_GP) * stride;
#pragma unroll
    for (int i = 0; i < 3; ++i) o[i * stride] = q[p].u[i];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) o[(3 + 3 * i + j) * stride] = q[p].G[i][j];
#pragma unroll
    for (int j = 0; j < 3; ++j) o[(12 + j) * stride] = q[p].gT[j];
#pragma unroll
    for (int i = 0; i < 3; ++i) o[(15 + i) * stride] = k.wtau * rM[i];
    o[18 * stride] = k.wtauT * rT;
  }
  cache[(long long)(8 * LIN_GP) * stride] = k.tau;
  cache[(long long)(8 * LIN_GP + 1) * stride] = k.tauT;
  cache[(long long)(8 * LIN_GP + 2) * stride] = k.alpha;
  cache[(long long)(8 * LIN_GP + 3) * stride] = k.K;
}

template <typename R>
NC_HD void elem_jvp_lin(const R* cache, long long stride, const R ue[3][8], const R ve[5][8],
                         R gam, R s, const ElemConst<R>& c, R out[5][8]) {
  const ElemCoef<R> k = lin_coef(cache, stride, gam, s, c);
  R uv = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) uv += ue[i][a] * ve[i][a];
  // the store holds wtau rM: the tangent takes dtau/tau = -tau^2 uv/16 (scaled units)
  const R rdtau = -k.tau * k.tau * R(0.0625) * uv;
  const R rdtauT = -k.tauT * k.tauT * R(0.0625) * uv;
  QP<R> d[8];
  interp_all8<R>(ve, d);
  R f0[8][5], F1[8][5][3];
#pragma unroll
  for (int P = 0; P < 4; ++P) {
    QP<R> q[2];
    R rM[2][3], rT[2];
    load_lin_pair<R>(cache, stride, P, q, rM, rT);
#pragma unroll
    for (int sx = 0; sx < 2; ++sx)
      flux_tangent_rm<R, false, true>(q[sx], rM[sx], rT[sx], d[2 * P + sx], k, R(0), R(0), rdtau,
                                      rdtauT, c, f0[2 * P + sx], F1[2 * P + sx]);
  }
  test_all8<R>(out, f0, F1, c.wc);
}

template <typename R>
NC_HD void elem_jtvp_lin(const R* cache, long long stride, const R ue[3][8], const R we[5][8],
                          R gam, R s, const ElemConst<R>& c, R out[5][8]) {
  const ElemCoef<R> k = lin_coef(cache, stride, gam, s, c);
  QP<R> t[8];
  interp_all8<R>(we, t);
  R f0[8][5], F1[8][5][3];
  R tb = R(0), tbT = R(0);
#pragma unroll
  for (int P = 0; P < 4; ++P) {
    QP<R> q[2];
    R rM[2][3], rT[2];
    load_lin_pair<R>(cache, stride, P, q, rM, rT);
#pragma unroll
    for (int sx = 0; sx < 2; ++sx)
      flux_adjoint_rm<R, true>(q[sx], rM[sx], rT[sx], t[2 * P + sx], k, c, f0[2 * P + sx],
                               F1[2 * P + sx], tb, tbT);
  }
  test_all8<R>(out, f0, F1, c.wc);
  // tb, tbT carry the store's factors wh tau, wh tauT: tau^3 tb wdt becomes tau^2 tb / 16
  const R gsum = -(k.tau * k.tau * tb + k.tauT * k.tauT * tbT) * R(0.0625);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) out[i][a] += gsum * ue[i][a];
}

// ---------------------------------------------------------------------------- element columns
// Pointwise tangent fluxes for a unit direction on one unknown of one node: phi
// = N_b and psi = grad N_b at the point, on unknown G (0-2 a velocity component,
// 3 the pressure, 4 the temperature).  The same terms as flux_tangent_rm with
// STORE (rM, rT the store's SUPG weights wtau rM, wtauT rT; whdtau, whdtauT the
// ratios dtau/tau, dtauT/tauT) with every product by a zero of the direction
// left out; the ratios are zero for G >= 3 (tau depends on the velocities only).
template <typename R, int G>
NC_HD void flux_column(const QP<R>& q, const R rM[3], R rT, R phi, const R psi[3],
                       const ElemCoef<R>& k, R whdtau, R whdtauT, const ElemConst<R>& c, R f0[5],
                       R F1[5][3]) {
  if (G < 3) {
    const R upsi = q.u[0] * psi[0] + q.u[1] * psi[1] + q.u[2] * psi[2];
    R a[3], b[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      R body = phi * q.G[i][G];  // d.u . grad u_i
      if (i == G) body += upsi + k.alpha * phi;
      f0[i] = body;
      a[i] = whdtau * rM[i] + k.wtau * body;
      b[i] = rM[i];
      F1[3][i] = a[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        R t = q.u[j] * a[i];
        if (i == j && i == G) t += c.prw2 * psi[i];
        if (i != j && i == G) t += c.prw * psi[j];
        if (i != j && j == G) t += c.prw * psi[i];
        if (j == G) t += phi * b[i];
        F1[i][j] = t;
      }
    const R drT = phi * q.gT[G];
    f0[3] = psi[G];
    f0[4] = drT;
    const R aT = whdtauT * rT + k.wtauT * drT, bT = rT;
#pragma unroll
    for (int j = 0; j < 3; ++j) F1[4][j] = j == G ? q.u[j] * aT + phi * bT : q.u[j] * aT;
  } else if (G == 3) {
    R a[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      f0[i] = R(0);
      a[i] = k.wtau * psi[i];
      F1[3][i] = a[i];
    }
    const R pw = c.wh * phi;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) F1[i][j] = i == j ? q.u[j] * a[i] - pw : q.u[j] * a[i];
    f0[3] = f0[4] = R(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) F1[4][j] = R(0);
  } else {
    R a[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const R body = c.beg[i] * phi;
      f0[i] = body;
      a[i] = k.wtau * body;
      F1[3][i] = a[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) F1[i][j] = q.u[j] * a[i];
    const R drT = q.u[0] * psi[0] + q.u[1] * psi[1] + q.u[2] * psi[2];
    f0[3] = R(0);
    f0[4] = drT;
    const R aT = k.wtauT * drT;
#pragma unroll
    for (int j = 0; j < 3; ++j) F1[4][j] = k.wK * psi[j] + q.u[j] * aT;
  }
}

// Column (b, G) of the element Jacobian from the linearisation store: the
// product elem_jvp_lin with the unit direction on unknown G of local node b.
// The direction's interpolation is N_b and grad N_b at the points in closed
// form (products of the 1-D weights), and flux_column forms only the nonzero
// tangent terms; the test side is the full one.
// ub: the state's velocity component G at node b (unused for G >= 3).
template <typename R, int G>
NC_HD void elem_column_lin(const R* cache, long long stride, R ub, int b, R gam, R s,
                           const ElemConst<R>& c, R out[5][8]) {
  const ElemCoef<R> k = lin_coef(cache, stride, gam, s, c);
  R whdtau = R(0), whdtauT = R(0);
  if (G < 3) {  // d(u_e^T u_e)/2 along the direction = u_e(G, b)
    // the store holds wtau rM: the ratio dtau/tau = -tau^2 ub/16 (scaled units)
    whdtau = -k.tau * k.tau * R(0.0625) * ub;
    whdtauT = -k.tauT * k.tauT * R(0.0625) * ub;
  }
  const R W[2] = {R(GW0), R(GW1)};  // weight of node bit 1 at point bit 0 / 1
  const int bx = b & 1, by = (b >> 1) & 1, bz = (b >> 2) & 1;
  const R sx = bx ? R(1) : R(-1), sy = by ? R(1) : R(-1), sz = bz ? R(1) : R(-1);
  R f0[8][5], F1[8][5][3];
#pragma unroll
  for (int P = 0; P < 4; ++P) {
    QP<R> q[2];
    R rM[2][3], rT[2];
    load_lin_pair<R>(cache, stride, P, q, rM, rT);
#pragma unroll
    for (int qx = 0; qx < 2; ++qx) {
      const int p = 2 * P + qx, qy = P & 1, qz = P >> 1;
      const R lx = bx ? W[qx] : R(1) - W[qx];
      const R ly = by ? W[qy] : R(1) - W[qy];
      const R lz = bz ? W[qz] : R(1) - W[qz];
      const R psi[3] = {sx * (ly * lz), sy * (lx * lz), sz * (lx * ly)};
      flux_column<R, G>(q[qx], rM[qx], rT[qx], lx * ly * lz, psi, k, whdtau, whdtauT, c, f0[p],
                        F1[p]);
    }
  }
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    if (G == 3 && f == 4) {  // the energy rows do not see the pressure
#pragma unroll
      for (int a = 0; a < 8; ++a) out[f][a] = R(0);
      continue;
    }
    R a0[8], b0[8][3];
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      a0[p] = f0[p][f];
      b0[p][0] = F1[p][f][0];
      b0[p][1] = F1[p][f][1];
      b0[p][2] = F1[p][f][2];
    }
    test8<R>(out[f], a0, b0, c.wc);
  }
}

template <typename R>
NC_HD ElemConst<R> make_const(double h, double Gr, double Pr, double amax, double qa, double qf,
                              double Ck, const double eg[3]) {
  ElemConst<R> c;
  c.inv_h = R(1.0 / h);
  c.wq = R((h / 2) * (h / 2) * (h / 2));
  c.wh = R((h / 2) * (h / 2) * (h / 2) / h);
  c.wc[0] = R((h / 2) * (h / 2) * (h / 2) / h * GW0);
  c.wc[1] = R((h / 2) * (h / 2) * (h / 2) / h * GW1);
  c.beg[0] = R(h * Gr * Pr * Pr * eg[0]);
  c.beg[1] = R(h * Gr * Pr * Pr * eg[1]);
  c.beg[2] = R(h * Gr * Pr * Pr * eg[2]);
  c.prw = R(Pr * (h / 2) * (h / 2) * (h / 2) / (h * h));
  c.prw2 = R(2.0 * Pr * (h / 2) * (h / 2) * (h / 2) / (h * h));
  c.h = R(h);
  c.prh = R(Pr / h);
  c.wdt = R((h / 2) * (h / 2) * (h / 2) / h / 16.0);
  c.iwh = R(h / ((h / 2) * (h / 2) * (h / 2)));
  c.t2s = R((4.0 * Pr / h) * (4.0 * Pr / h));
  c.amax = R(amax);
  c.qa = R(qa);
  c.qf = R(qf);
  c.Ck = R(Ck);
  return c;
}

}  // namespace nc
