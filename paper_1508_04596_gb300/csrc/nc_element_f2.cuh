// FP32 element products J v and J^T w on packed pairs (two FP32 values per
// 64-bit register pair, one add / sub / mul / fma .f32x2 instruction for both).
//
// The FP32 element kernels are bound by instruction issue, not by the FMA pipe
// (about half of the issue slots go to FP32 instructions while the pipe is half
// busy).  A packed instruction does two lanes' worth of FP32 arithmetic in one
// issue slot, so the same arithmetic as elem_jvp / elem_jtvp is reorganised on
// pairs:
//  * interpolation (the tensor-product stages of interp8): the z and y stages
//    act on node pairs along x (local nodes a, a + 1); the x stage, which mixes
//    the two nodes of a pair into the two Gauss points qx = 0, 1, is scalar and
//    leaves its results as point pairs;
//  * pointwise fluxes on point pairs (qx = 0, 1 at fixed qy, qz): every
//    operation of flux_tangent_rm / flux_adjoint_rm is the same for both points,
//    with the element coefficients broadcast to both lanes;
//  * the test side (test8) mirrors the interpolation: a scalar x stage from
//    point pairs to node pairs, then packed y and z stages.
// The result equals elem_jvp<float> / elem_jtvp<float> up to FP32 rounding
// (different order of some sums); the host check compares them.
//
// Pair index P = qy + 2 qz of the four point pairs, lanes .x / .y = qx 0 / 1.
// Node pairs: NP[ja + 2 ka] = (node ia = 0, node ia = 1).
#pragma once
#include <cstring>

#include "nc_element.cuh"

namespace nc {

#if defined(__CUDACC__)
typedef float2 f2;
NC_HD f2 mk2(float a, float b) { return make_float2(a, b); }
#else
struct f2 {
  float x, y;
};
inline f2 mk2(float a, float b) { return f2{a, b}; }
#endif

NC_HD f2 bc2(float s) { return mk2(s, s); }

NC_HD f2 add2(f2 a, f2 b) {
#if defined(__CUDA_ARCH__)
  return __fadd2_rn(a, b);
#else
  return mk2(a.x + b.x, a.y + b.y);
#endif
}
NC_HD f2 sub2(f2 a, f2 b) {
#if defined(__CUDA_ARCH__)
  unsigned long long ra, rb, rr;
  memcpy(&ra, &a, 8);
  memcpy(&rb, &b, 8);
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rr) : "l"(ra), "l"(rb));
  f2 r;
  memcpy(&r, &rr, 8);
  return r;
#else
  return mk2(a.x - b.x, a.y - b.y);
#endif
}
NC_HD f2 mul2(f2 a, f2 b) {
#if defined(__CUDA_ARCH__)
  return __fmul2_rn(a, b);
#else
  return mk2(a.x * b.x, a.y * b.y);
#endif
}
// a * b + c, one rounding per lane
NC_HD f2 fma2(f2 a, f2 b, f2 c) {
#if defined(__CUDA_ARCH__)
  return __ffma2_rn(a, b, c);
#else
  return mk2(std::fma(a.x, b.x, c.x), std::fma(a.y, b.y, c.y));
#endif
}
NC_HD f2 neg2(f2 a) { return mk2(-a.x, -a.y); }

// Quadrature-point state of a point pair.
struct QP2 {
  f2 u[3], G[3][3], p, gp[3], T, gT[3];
};

// Element coefficients broadcast to both lanes (from ElemCoef<float>).
struct Coef2 {
  f2 alpha, K, tau, tauT, s, wtau, wtauT, wK;
};

NC_HD Coef2 coef2(const ElemCoef<float>& k) {
  Coef2 b;
  b.alpha = bc2(k.alpha);
  b.K = bc2(k.K);
  b.tau = bc2(k.tau);
  b.tauT = bc2(k.tauT);
  b.s = bc2(k.s);
  b.wtau = bc2(k.wtau);
  b.wtauT = bc2(k.wtauT);
  b.wK = bc2(k.wK);
  return b;
}

// Kernel-wide constants broadcast to both lanes (from ElemConst<float>).
struct Const2 {
  f2 wq, wh, Pr, prw, prw2, beg[3], c[2], two;  // Pr: Pr/h (reference gradients)
};

NC_HD Const2 const2(const ElemConst<float>& c) {
  Const2 b;
  b.wq = bc2(c.wq);
  b.wh = bc2(c.wh);
  b.Pr = bc2(c.prh);
  b.prw = bc2(c.prw);
  b.prw2 = bc2(c.prw2);
  for (int i = 0; i < 3; ++i) b.beg[i] = bc2(c.beg[i]);
  b.c[0] = bc2(float(GW0));
  b.c[1] = bc2(float(GW1));
  b.two = bc2(2.0f);
  return b;
}

// ------------------------------------------------------------------ interpolation
// Values and reference gradients (h grad) of one Q1 field at the 8 Gauss points,
// as point pairs: val[P], g[P][j].
NC_HD void interp8_f2(const float x[8], const Const2& K, f2 val[4], f2 g[4][3]) {
  const float c[2] = {float(GW0), float(GW1)};
  // node pairs along x: X[ja][ka]
  const f2 X00 = mk2(x[0], x[1]), X10 = mk2(x[2], x[3]);
  const f2 X01 = mk2(x[4], x[5]), X11 = mk2(x[6], x[7]);
  // z stage: differences and values at both qz, per ja
  const f2 DZ0 = sub2(X01, X00), DZ1 = sub2(X11, X10);
  f2 VZ[2][2];
#pragma unroll
  for (int qz = 0; qz < 2; ++qz) {
    VZ[qz][0] = fma2(K.c[qz], DZ0, X00);
    VZ[qz][1] = fma2(K.c[qz], DZ1, X10);
  }
  // y stage: differences and values at both qy, per qz; the z difference
  // interpolated in y
  f2 DY[2], VYZ[2][2];
#pragma unroll
  for (int qz = 0; qz < 2; ++qz) {
    DY[qz] = sub2(VZ[qz][1], VZ[qz][0]);
    VYZ[qz][0] = fma2(K.c[0], DY[qz], VZ[qz][0]);
    VYZ[qz][1] = fma2(K.c[1], DY[qz], VZ[qz][0]);
  }
  const f2 EZ = sub2(DZ1, DZ0);
  const f2 DZY[2] = {fma2(K.c[0], EZ, DZ0), fma2(K.c[1], EZ, DZ0)};
  // x stage: the two nodes of a pair -> the two points of a pair
#pragma unroll
  for (int qz = 0; qz < 2; ++qz)
#pragma unroll
    for (int qy = 0; qy < 2; ++qy) {
      const int P = qy + 2 * qz;
      const f2 v = VYZ[qz][qy];
      const float dx = v.y - v.x;
      val[P] = mk2(v.x + c[0] * dx, v.x + c[1] * dx);
      g[P][0] = mk2(dx, dx);
    }
#pragma unroll
  for (int qz = 0; qz < 2; ++qz) {
    const float ey = DY[qz].y - DY[qz].x;
    const f2 gy = mk2(DY[qz].x + c[0] * ey, DY[qz].x + c[1] * ey);
    g[2 * qz][1] = gy;
    g[1 + 2 * qz][1] = gy;
  }
#pragma unroll
  for (int qy = 0; qy < 2; ++qy) {
    const float ex = DZY[qy].y - DZY[qy].x;
    const f2 gz = mk2(DZY[qy].x + c[0] * ex, DZY[qy].x + c[1] * ex);
    g[qy][2] = gz;
    g[qy + 2][2] = gz;
  }
}

NC_HD void interp_all_f2(const float xe[5][8], const Const2& K, QP2 q[4]) {
  f2 val[4], g[4][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    interp8_f2(xe[i], K, val, g);
#pragma unroll
    for (int P = 0; P < 4; ++P) {
      q[P].u[i] = val[P];
      q[P].G[i][0] = g[P][0];
      q[P].G[i][1] = g[P][1];
      q[P].G[i][2] = g[P][2];
    }
  }
  interp8_f2(xe[3], K, val, g);
#pragma unroll
  for (int P = 0; P < 4; ++P) {
    q[P].p = val[P];
    q[P].gp[0] = g[P][0];
    q[P].gp[1] = g[P][1];
    q[P].gp[2] = g[P][2];
  }
  interp8_f2(xe[4], K, val, g);
#pragma unroll
  for (int P = 0; P < 4; ++P) {
    q[P].T = val[P];
    q[P].gT[0] = g[P][0];
    q[P].gT[1] = g[P][1];
    q[P].gT[2] = g[P][2];
  }
}

// ------------------------------------------------------------------ test side
// Transpose of interp8_f2 (reference gradients, as in test8): out[a] =
// sum_p [w N_a(p) f0[p] + dN_a/dxi_j(p) F1[p][j]] (test8, with the value slots'
// Gauss weight applied here, wc = (w/h) (1 -+ 1/sqrt 3)/2), with f0, F1 as point
// pairs and out as node pairs out[ja + 2 ka] = (out[a], out[a + 1]).
NC_HD void test8_f2(f2 out[4], const f2 f0[4], const f2 F1[4][3], const float wc[2],
                    const Const2& K) {
  const float c[2] = {float(GW0), float(GW1)};
  // x stage: point pairs -> node pairs
  f2 VYZB[2][2];
#pragma unroll
  for (int qz = 0; qz < 2; ++qz)
#pragma unroll
    for (int qy = 0; qy < 2; ++qy) {
      const int P = qy + 2 * qz;
      const f2 f = f0[P], Fp = F1[P][0];
      const float F = Fp.x + Fp.y;
      VYZB[qz][qy] = mk2(wc[1] * f.x + (wc[0] * f.y - F), wc[0] * f.x + (wc[1] * f.y + F));
    }
  f2 DYB[2];
#pragma unroll
  for (int qz = 0; qz < 2; ++qz) {
    const f2 b = add2(F1[2 * qz][1], F1[1 + 2 * qz][1]);  // (qx = 0, qx = 1), summed over qy
    const float eyb = c[0] * b.x + c[1] * b.y;
    DYB[qz] = mk2(b.x + b.y - eyb, eyb);
  }
  f2 DZYB[2];
#pragma unroll
  for (int qy = 0; qy < 2; ++qy) {
    const f2 b = add2(F1[qy][2], F1[qy + 2][2]);  // summed over qz
    const float exb = c[0] * b.x + c[1] * b.y;
    DZYB[qy] = mk2(b.x + b.y - exb, exb);
  }
  // y stage on node pairs
  f2 VZB[2][2];
#pragma unroll
  for (int qz = 0; qz < 2; ++qz) {
    const f2 d = fma2(K.c[1], VYZB[qz][1], fma2(K.c[0], VYZB[qz][0], DYB[qz]));
    VZB[qz][0] = sub2(add2(VYZB[qz][0], VYZB[qz][1]), d);
    VZB[qz][1] = d;
  }
  const f2 ezb = fma2(K.c[1], DZYB[1], mul2(K.c[0], DZYB[0]));
  const f2 DZB[2] = {sub2(add2(DZYB[0], DZYB[1]), ezb), ezb};
  // z stage on node pairs
#pragma unroll
  for (int ja = 0; ja < 2; ++ja) {
    const f2 d = fma2(K.c[1], VZB[1][ja], fma2(K.c[0], VZB[0][ja], DZB[ja]));
    out[ja] = sub2(add2(VZB[0][ja], VZB[1][ja]), d);
    out[ja + 2] = d;
  }
}

NC_HD void test_all_f2(float out[5][8], const f2 f0[4][5], const f2 F1[4][5][3],
                       const float wc[2], const Const2& K) {
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    f2 a[4], b[4][3], o[4];
#pragma unroll
    for (int P = 0; P < 4; ++P) {
      a[P] = f0[P][f];
      b[P][0] = F1[P][f][0];
      b[P][1] = F1[P][f][1];
      b[P][2] = F1[P][f][2];
    }
    test8_f2(o, a, b, wc, K);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      out[f][2 * n] = o[n].x;
      out[f][2 * n + 1] = o[n].y;
    }
  }
}

// ------------------------------------------------------------------ fluxes
// Strong residuals of a point pair (strong()).
NC_HD void strong_f2(const QP2& q, const Coef2& k, const Const2& K, f2 body[3], f2 rM[3], f2& rT) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    body[i] = fma2(q.u[0], q.G[i][0],
                   fma2(q.u[1], q.G[i][1],
                        fma2(q.u[2], q.G[i][2], fma2(k.alpha, q.u[i], mul2(K.beg[i], q.T)))));
    rM[i] = add2(body[i], q.gp[i]);
  }
  rT = fma2(q.u[0], q.gT[0], fma2(q.u[1], q.gT[1], fma2(q.u[2], q.gT[2], neg2(k.s))));
}

// Tangent fluxes of a point pair in the state direction d (flux_tangent_rm
// without the parameter directions): f0 without the Gauss weight (applied on the
// test side) and (w/h)-scaled F1.
NC_HD void flux_tangent_f2(const QP2& q, const f2 rM[3], f2 rT, const QP2& d, const Coef2& k,
                           f2 whdtau, f2 whdtauT, const Const2& K, f2 f0[5], f2 F1[5][3]) {
  f2 a[3], b[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    f2 body = mul2(d.u[0], q.G[i][0]);
    body = fma2(d.u[1], q.G[i][1], body);
    body = fma2(d.u[2], q.G[i][2], body);
    body = fma2(q.u[0], d.G[i][0], body);
    body = fma2(q.u[1], d.G[i][1], body);
    body = fma2(q.u[2], d.G[i][2], body);
    body = fma2(k.alpha, d.u[i], body);
    body = fma2(K.beg[i], d.T, body);
    const f2 drM = add2(body, d.gp[i]);
    f0[i] = body;
    a[i] = fma2(whdtau, rM[i], mul2(k.wtau, drM));
    b[i] = mul2(k.wtau, rM[i]);
    F1[3][i] = a[i];
  }
  // viscous part once per symmetric pair, pressure on the diagonal
  const f2 pw = mul2(K.wh, d.p);
  const f2 v01 = mul2(K.prw, add2(d.G[0][1], d.G[1][0]));
  const f2 v02 = mul2(K.prw, add2(d.G[0][2], d.G[2][0]));
  const f2 v12 = mul2(K.prw, add2(d.G[1][2], d.G[2][1]));
  const f2 vd[3] = {fma2(K.prw2, d.G[0][0], neg2(pw)), fma2(K.prw2, d.G[1][1], neg2(pw)),
                    fma2(K.prw2, d.G[2][2], neg2(pw))};
  const f2 vo[3][3] = {{vd[0], v01, v02}, {v01, vd[1], v12}, {v02, v12, vd[2]}};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) F1[i][j] = fma2(d.u[j], b[i], fma2(q.u[j], a[i], vo[i][j]));
  f2 drT = mul2(d.u[0], q.gT[0]);
  drT = fma2(d.u[1], q.gT[1], drT);
  drT = fma2(d.u[2], q.gT[2], drT);
  drT = fma2(q.u[0], d.gT[0], drT);
  drT = fma2(q.u[1], d.gT[1], drT);
  drT = fma2(q.u[2], d.gT[2], drT);
  f0[3] = add2(add2(d.G[0][0], d.G[1][1]), d.G[2][2]);
  f0[4] = drT;
  const f2 aT = fma2(whdtauT, rT, mul2(k.wtauT, drT)), bT = mul2(k.wtauT, rT);
#pragma unroll
  for (int j = 0; j < 3; ++j) F1[4][j] = fma2(d.u[j], bT, fma2(q.u[j], aT, mul2(k.wK, d.gT[j])));
}

// Cotangent fluxes of a point pair for the test field t (flux_adjoint_rm):
// f0 (value slots, without the Gauss weight) and F1 (gradient slots,
// (w/h)-scaled); the
// cotangents of tau and tau_T are accumulated per lane, without the weight.
NC_HD void flux_adjoint_f2(const QP2& q, const f2 rM[3], f2 rT, const QP2& t, const Coef2& k,
                           const Const2& K, f2 f0[5], f2 F1[5][3], f2& tau_bar, f2& tauT_bar) {
  const f2* const C1[5] = {t.G[0], t.G[1], t.G[2], t.gp, t.gT};
  const f2 c0[5] = {t.u[0], t.u[1], t.u[2], t.p, t.T};
  f2 rMb[3], ub[3], Gb[3][3], gTb[3];
  const f2 C4u = fma2(C1[4][0], q.u[0], fma2(C1[4][1], q.u[1], mul2(C1[4][2], q.u[2])));
  const f2 rTb = fma2(k.tauT, C4u, c0[4]);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const f2 s = fma2(C1[i][0], q.u[0], fma2(C1[i][1], q.u[1], fma2(C1[i][2], q.u[2], C1[3][i])));
    rMb[i] = mul2(k.tau, s);
    tau_bar = fma2(s, rM[i], tau_bar);
  }
  tauT_bar = fma2(C4u, rT, tauT_bar);
  const f2 pb = neg2(add2(add2(C1[0][0], C1[1][1]), C1[2][2]));
  f2 Tb = mk2(0.0f, 0.0f);
  const f2 trT = mul2(k.tauT, rT);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const f2 m = fma2(C1[0][j], rM[0], fma2(C1[1][j], rM[1], mul2(C1[2][j], rM[2])));
    ub[j] = fma2(rTb, q.gT[j], fma2(C1[4][j], trT, mul2(k.tau, m)));
    gTb[j] = fma2(rTb, q.u[j], mul2(k.K, C1[4][j]));
  }
  {
    const f2 g01 = mul2(K.Pr, add2(C1[0][1], C1[1][0]));
    const f2 g02 = mul2(K.Pr, add2(C1[0][2], C1[2][0]));
    const f2 g12 = mul2(K.Pr, add2(C1[1][2], C1[2][1]));
    const f2 p2x = mul2(K.two, K.Pr);
    Gb[0][0] = fma2(p2x, C1[0][0], c0[3]);
    Gb[1][1] = fma2(p2x, C1[1][1], c0[3]);
    Gb[2][2] = fma2(p2x, C1[2][2], c0[3]);
    Gb[0][1] = Gb[1][0] = g01;
    Gb[0][2] = Gb[2][0] = g02;
    Gb[1][2] = Gb[2][1] = g12;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const f2 cb = add2(c0[i], rMb[i]);  // cotangent of conv_i (and of the body terms)
    ub[i] = fma2(k.alpha, cb, ub[i]);
    Tb = fma2(K.beg[i], cb, Tb);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ub[j] = fma2(cb, q.G[i][j], ub[j]);
      Gb[i][j] = fma2(cb, q.u[j], Gb[i][j]);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    f0[i] = ub[i];
    F1[i][0] = mul2(K.wh, Gb[i][0]);
    F1[i][1] = mul2(K.wh, Gb[i][1]);
    F1[i][2] = mul2(K.wh, Gb[i][2]);
    F1[3][i] = mul2(K.wh, rMb[i]);
    F1[4][i] = mul2(K.wh, gTb[i]);
  }
  f0[3] = pb;
  f0[4] = Tb;
}

// ------------------------------------------------------------------ element products
// J v of one element (elem_jvp<float> on point pairs).
NC_HD void elem_jvp_f2(const float xe[5][8], const float ve[5][8], float gam, float s,
                       const ElemConst<float>& c, float out[5][8]) {
  float S;
  const ElemCoef<float> ks = elem_coef(xe, gam, s, c, S);
  float uv = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) uv += xe[i][a] * ve[i][a];
  const float dtau = -ks.tau * ks.tau * ks.tau * 0.0625f * uv;  // scaled units (elem_jvp)
  const float dtauT = -ks.tauT * ks.tauT * ks.tauT * 0.0625f * uv;
  const Const2 K = const2(c);
  const Coef2 k = coef2(ks);
  const f2 whdtau = bc2(c.wh * dtau), whdtauT = bc2(c.wh * dtauT);
  QP2 q[4], d[4];
  interp_all_f2(xe, K, q);
  interp_all_f2(ve, K, d);
  f2 f0[4][5], F1[4][5][3];
#pragma unroll
  for (int P = 0; P < 4; ++P) {
    f2 body[3], rM[3], rT;
    strong_f2(q[P], k, K, body, rM, rT);
    flux_tangent_f2(q[P], rM, rT, d[P], k, whdtau, whdtauT, K, f0[P], F1[P]);
  }
  test_all_f2(out, f0, F1, c.wc, K);
}

// J^T w of one element (elem_jtvp<float> on point pairs).
NC_HD void elem_jtvp_f2(const float xe[5][8], const float we[5][8], float gam, float s,
                        const ElemConst<float>& c, float out[5][8]) {
  float S;
  const ElemCoef<float> ks = elem_coef(xe, gam, s, c, S);
  const Const2 K = const2(c);
  const Coef2 k = coef2(ks);
  QP2 q[4], t[4];
  interp_all_f2(xe, K, q);
  interp_all_f2(we, K, t);
  f2 f0[4][5], F1[4][5][3];
  f2 tb = mk2(0.0f, 0.0f), tbT = mk2(0.0f, 0.0f);
#pragma unroll
  for (int P = 0; P < 4; ++P) {
    f2 body[3], rM[3], rT;
    strong_f2(q[P], k, K, body, rM, rT);
    flux_adjoint_f2(q[P], rM, rT, t[P], k, K, f0[P], F1[P], tb, tbT);
  }
  test_all_f2(out, f0, F1, c.wc, K);
  const float tbs = tb.x + tb.y, tbTs = tbT.x + tbT.y;
  const float gsum = -(ks.tau * ks.tau * ks.tau * tbs + ks.tauT * ks.tauT * ks.tauT * tbTs) * c.wdt;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int a = 0; a < 8; ++a) out[i][a] += gsum * xe[i][a];
}

}  // namespace nc
