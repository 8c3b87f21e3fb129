// PDE (Helmholtz) density filter (Sec. 3.2; filter radius 2.5 h in Sec. 6.3-6.4).
//
//   -r^2 lap(rho~) + rho~ = rho,  Neumann boundary,  r = R / (2 sqrt 3),
//
// with trilinear nodal rho~, element-constant rho, and the filtered element
// value the mean of its eight nodes: gamma~ = P rho, P = h^-3 T^T (r^2 K + M)^-1 T,
// T_{n,e} = int_e N_n = h^3/8.  P is symmetric, so the same call applies the
// chain rule dPhi/drho = P dPhi/dgamma~.
//
// On a uniform grid every element matrix is the same, so r^2 K + M is applied
// node by node as a sum over the node's (up to 8) elements of the closed-form
// Q1 entries (stiffness h/3, 0, -h/12, -h/12 and mass h^3/216 * 2^(shared
// coordinates), by the number of coordinates in which the two corners differ).
// The SPD system is solved by Jacobi-preconditioned conjugate gradients in FP64.
#include <cmath>

#include "nc_internal.cuh"

namespace nc {
nc_status set_err(nc_ctx* ctx, nc_status st, const std::string& msg);
nc_status cuda_check(nc_ctx* ctx, cudaError_t e, const char* what);
}  // namespace nc

using namespace nc;

namespace {

constexpr int FT = 256;

inline unsigned fblocks(long long n) { return (unsigned)((n + FT - 1) / FT); }

struct HelmCoef {
  double A[4];  // entry of r^2 K_e + M_e by the number of differing coordinates
};

HelmCoef helm_coef(double h, double R) {
  const double r2 = R * R / 12.0;
  const double K[4] = {h / 3.0, 0.0, -h / 12.0, -h / 12.0};
  const double M[4] = {8.0, 4.0, 2.0, 1.0};
  HelmCoef c;
  for (int q = 0; q < 4; ++q) c.A[q] = r2 * K[q] + M[q] * h * h * h / 216.0;
  return c;
}

// y = (r^2 K + M) x, one thread per node; diag receives the diagonal if not null.
__global__ void k_helm_apply(LevelDev d, HelmCoef c, const double* __restrict__ x,
                             double* __restrict__ y, double* __restrict__ diag) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= d.Nn) return;
  int i, j, k;
  node_ijk(d, n, i, j, k);
  const long long sy = d.nx + 1, sz = (long long)(d.nx + 1) * (d.ny + 1);
  double acc = 0.0, dg = 0.0;
  for (int a = 0; a < 8; ++a) {  // the node is local corner a of element (i-ia, j-ja, k-ka)
    const int ia = a & 1, ja = (a >> 1) & 1, ka = (a >> 2) & 1;
    const int ie = i - ia, je = j - ja, ke = k - ka;
    if (ie < 0 || je < 0 || ke < 0 || ie >= d.nx || je >= d.ny || ke >= d.nz) continue;
    const long long n0 = ie + sy * (je + (long long)(d.ny + 1) * ke);
    for (int b = 0; b < 8; ++b) {
      const long long m = n0 + (b & 1) + ((b >> 1) & 1) * sy + ((b >> 2) & 1) * sz;
      acc += c.A[__popc(a ^ b)] * (x ? x[m] : 0.0);
    }
    dg += c.A[0];
  }
  if (y) y[n] = acc;
  if (diag) diag[n] = dg;
}

// b_n = sum over the node's elements of rho_e h^3 / 8
__global__ void k_helm_rhs(LevelDev d, const double* __restrict__ rho, double* __restrict__ b) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= d.Nn) return;
  int i, j, k;
  node_ijk(d, n, i, j, k);
  double acc = 0.0;
  for (int a = 0; a < 8; ++a) {
    const int ie = i - (a & 1), je = j - ((a >> 1) & 1), ke = k - ((a >> 2) & 1);
    if (ie < 0 || je < 0 || ke < 0 || ie >= d.nx || je >= d.ny || ke >= d.nz) continue;
    acc += rho[ie + (long long)d.nx * (je + (long long)d.ny * ke)];
  }
  b[n] = acc * d.h * d.h * d.h * 0.125;
}

// gamma~_e = mean of the element's eight nodal values
__global__ void k_elem_mean(LevelDev d, const double* __restrict__ x, double* __restrict__ g) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  int i, j, k;
  elem_ijk(d, e, i, j, k);
  const long long sy = d.nx + 1, sz = (long long)(d.nx + 1) * (d.ny + 1);
  const long long n0 = i + sy * (j + (long long)(d.ny + 1) * k);
  double acc = 0.0;
  for (int a = 0; a < 8; ++a) acc += x[n0 + (a & 1) + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz];
  g[e] = 0.125 * acc;
}

nc_status dot(nc_ctx* ctx, long long n, const double* a, const double* b, double* out,
              cudaStream_t s) {
  vmdot(n, 1, a, 0, b, ctx->dscal, ctx->partial, s);
  nc_status st = cuda_check(ctx, cudaMemcpyAsync(out, ctx->dscal, sizeof(double),
                                                 cudaMemcpyDeviceToHost, s), "filter dot");
  if (st != NC_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(s), "filter sync");
}

}  // namespace

extern "C" nc_status nc_filter(nc_ctx* ctx, const double* rho, double* gamma_f, double radius,
                               void* stream) {
  if (!ctx || !rho || !gamma_f || !(radius >= 0.0) || !std::isfinite(radius))
    return set_err(ctx, NC_ERR_ARG, "nc_filter: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const Level& L = ctx->lv[0];
  const LevelDev& d = L.d;
  const long long Nn = d.Nn;
  nc_status st;
  for (int q = 0; q < 6; ++q)
    if (!ctx->filt[q] &&
        (st = cuda_check(ctx, cudaMalloc((void**)&ctx->filt[q], sizeof(double) * Nn),
                         "cudaMalloc filter")) != NC_OK)
      return st;
  double *x = ctx->filt[0], *r = ctx->filt[1], *z = ctx->filt[2], *p = ctx->filt[3],
         *q = ctx->filt[4], *dg = ctx->filt[5];
  const HelmCoef c = helm_coef(d.h, radius);
  k_helm_apply<<<fblocks(Nn), FT, 0, s>>>(d, c, nullptr, nullptr, dg);
  k_helm_rhs<<<fblocks(Nn), FT, 0, s>>>(d, rho, r);  // r = b (x = 0)
  vzero(Nn, x, s);
  double bb, rz, pq, rr;
  if ((st = dot(ctx, Nn, r, r, &bb, s)) != NC_OK) return st;
  if (!std::isfinite(bb)) return set_err(ctx, NC_ERR_NAN, "nc_filter: non-finite design");
  const double tol2 = 1e-26 * bb;  // ||r|| <= 1e-13 ||b||
  if (bb > 0.0) {
    vdiv(Nn, (const double*)r, (const double*)dg, z, s);
    vcopy(Nn, (const double*)z, p, s);
    if ((st = dot(ctx, Nn, r, z, &rz, s)) != NC_OK) return st;
    int it = 0;
    for (; it < 1000; ++it) {
      k_helm_apply<<<fblocks(Nn), FT, 0, s>>>(d, c, p, q, nullptr);
      if ((st = dot(ctx, Nn, p, q, &pq, s)) != NC_OK) return st;
      if (!(pq > 0.0)) break;
      const double alpha = rz / pq;
      vaxpy(Nn, alpha, (const double*)p, x, s);
      vaxpy(Nn, -alpha, (const double*)q, r, s);
      if ((st = dot(ctx, Nn, r, r, &rr, s)) != NC_OK) return st;
      if (rr <= tol2) break;
      vdiv(Nn, (const double*)r, (const double*)dg, z, s);
      double rz_new;
      if ((st = dot(ctx, Nn, r, z, &rz_new, s)) != NC_OK) return st;
      vxpay(Nn, (const double*)z, rz_new / rz, p, s);  // p = z + beta p
      rz = rz_new;
    }
    if (it >= 1000) return set_err(ctx, NC_ERR_MAXIT, "nc_filter: CG did not converge");
  }
  k_elem_mean<<<fblocks(d.E), FT, 0, s>>>(d, x, gamma_f);
  return cuda_check(ctx, cudaStreamSynchronize(s), "nc_filter");
}
