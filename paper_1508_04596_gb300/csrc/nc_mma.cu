// Design update of the optimisation problem (Sec. 3.2): the volume constraint
// and one iteration of the method of moving asymptotes (MMA, Svanberg 1987)
// for one inequality constraint.
//
// MMA as implemented (the paper names the method and prints no details):
//  * asymptotes: iterations 0 and 1 put L, U at x -/+ 0.5 (xmax - xmin); later
//    ones widen them by 1.2 where a variable moved the same way twice, narrow
//    them by 0.7 where it oscillated, and keep them within 0.01 .. 10 times
//    (xmax - xmin) of x;
//  * move limits: alpha = max(xmin, L + 0.1 (x - L), x - move d),
//    beta = min(xmax, U - 0.1 (U - x), x + move d), d = xmax - xmin;
//  * each function f_i (objective, constraint) is replaced by the separable
//    convex approximation with p = (U - x)^2 (1.001 a+ + 0.001 a- + 1e-5 / d),
//    q = (x - L)^2 (0.001 a+ + 1.001 a- + 1e-5 / d), a = df_i/dx_j;
//  * the subproblem is solved through its dual: for a multiplier lam the
//    minimiser of the Lagrangian is, per variable, the clipped
//    (L sqrt(P) + U sqrt(Q)) / (sqrt(P) + sqrt(Q)), P = p0 + lam p1,
//    Q = q0 + lam q1, and the approximated constraint does not increase with
//    lam; lam = 0 if it already holds, else the host brackets lam by doubling
//    from 1 and bisects to floating-point resolution.  Every evaluation of the
//    approximated constraint is one pass over the variables (fixed-partition
//    reduction, deterministic).
#include <cmath>

#include "nc_internal.cuh"

namespace nc {
nc_status set_err(nc_ctx* ctx, nc_status st, const std::string& msg);
nc_status cuda_check(nc_ctx* ctx, cudaError_t e, const char* what);
}  // namespace nc

using namespace nc;

namespace {

constexpr int MT = 256;
constexpr int MMA_BLOCKS = 304;  // 2 x 152 SMs: fixed reduction partition

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Block sum (or maximum) of one value per thread -> partial[blockIdx.x].
template <bool MAX>
__device__ __forceinline__ void block_partial(double v, double* partial) {
  __shared__ double sh[MT / 32];
  v = MAX ? warp_max_d(v) : warp_sum_d(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < MT / 32 ? sh[lane] : 0.0;
    v = MAX ? warp_max_d(v) : warp_sum_d(v);
    if (lane == 0) partial[blockIdx.x] = v;
  }
}

// Fold the partials in index order (one block).
__global__ void __launch_bounds__(MT) k_fold(int nb, const double* partial, double* out) {
  __shared__ double sh[MT / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += MT) v += partial[b];
  v = warp_sum_d(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < MT / 32 ? sh[lane] : 0.0;
    v = warp_sum_d(v);
    if (lane == 0) *out = v;
  }
}

// partial sums of (1 - gamma_e) and of the active count over the variables
__global__ void __launch_bounds__(MT) k_volume(long long n, const double* __restrict__ g,
                                               const unsigned char* __restrict__ active,
                                               double* partial, double* partial_cnt) {
  double acc = 0.0, cnt = 0.0;
  for (long long j = blockIdx.x * (long long)MT + threadIdx.x; j < n; j += (long long)gridDim.x * MT) {
    if (active && !active[j]) continue;
    acc += 1.0 - g[j];
    cnt += 1.0;
  }
  block_partial<false>(acc, partial);
  __syncthreads();
  block_partial<false>(cnt, partial_cnt);
}

__global__ void k_volume_grad(long long n, const unsigned char* __restrict__ active, double dgval,
                              double* __restrict__ dg) {
  const long long j = blockIdx.x * (long long)MT + threadIdx.x;
  if (j >= n) return;
  dg[j] = (!active || active[j]) ? dgval : 0.0;
}

// Asymptotes of iteration k, in place.
__global__ void k_mma_asym(long long n, int k, const double* __restrict__ x,
                           const double* __restrict__ xo1, const double* __restrict__ xo2,
                           double* __restrict__ low, double* __restrict__ upp,
                           const unsigned char* __restrict__ active, double xmin, double xmax) {
  const long long j = blockIdx.x * (long long)MT + threadIdx.x;
  if (j >= n || (active && !active[j])) return;
  const double d = xmax - xmin, xj = x[j];
  if (k < 2) {
    low[j] = xj - 0.5 * d;
    upp[j] = xj + 0.5 * d;
    return;
  }
  const double s = (xj - xo1[j]) * (xo1[j] - xo2[j]);
  const double fac = s < 0.0 ? 0.7 : (s > 0.0 ? 1.2 : 1.0);
  double l = xj - fac * (xo1[j] - low[j]);
  double u = xj + fac * (upp[j] - xo1[j]);
  l = fmin(fmax(l, xj - 10.0 * d), xj - 0.01 * d);
  u = fmin(fmax(u, xj + 0.01 * d), xj + 10.0 * d);
  low[j] = l;
  upp[j] = u;
}

struct MmaVar {
  double y, f1_term;
};

// Minimiser y_j(lam) of the separable Lagrangian and its term of the
// approximated constraint.
__device__ __forceinline__ MmaVar mma_var(double xj, double l, double u, double a0, double a1,
                                          double lam, double xmin, double xmax, double move) {
  const double d = xmax - xmin, r = 1e-5 / d;
  const double a0p = fmax(a0, 0.0), a0m = fmax(-a0, 0.0);
  const double a1p = fmax(a1, 0.0), a1m = fmax(-a1, 0.0);
  const double ux2 = (u - xj) * (u - xj), xl2 = (xj - l) * (xj - l);
  const double p0 = ux2 * (1.001 * a0p + 0.001 * a0m + r), q0 = xl2 * (0.001 * a0p + 1.001 * a0m + r);
  const double p1 = ux2 * (1.001 * a1p + 0.001 * a1m + r), q1 = xl2 * (0.001 * a1p + 1.001 * a1m + r);
  const double alpha = fmax(fmax(xmin, l + 0.1 * (xj - l)), xj - move * d);
  const double beta = fmin(fmin(xmax, u - 0.1 * (u - xj)), xj + move * d);
  const double sP = sqrt(p0 + lam * p1), sQ = sqrt(q0 + lam * q1);
  const double y = fmin(fmax((l * sP + u * sQ) / (sP + sQ), alpha), beta);
  MmaVar v;
  v.y = y;
  v.f1_term = p1 * (1.0 / (u - y) - 1.0 / (u - xj)) + q1 * (1.0 / (y - l) - 1.0 / (xj - l));
  return v;
}

__global__ void __launch_bounds__(MT) k_mma_dual(long long n, const double* __restrict__ x,
                                                 const double* __restrict__ low,
                                                 const double* __restrict__ upp,
                                                 const double* __restrict__ df0,
                                                 const double* __restrict__ df1,
                                                 const unsigned char* __restrict__ active,
                                                 double lam, double xmin, double xmax, double move,
                                                 double scale0, double* partial) {
  double acc = 0.0;
  for (long long j = blockIdx.x * (long long)MT + threadIdx.x; j < n; j += (long long)gridDim.x * MT) {
    if (active && !active[j]) continue;
    acc += mma_var(x[j], low[j], upp[j], scale0 * df0[j], df1[j], lam, xmin, xmax, move).f1_term;
  }
  block_partial<false>(acc, partial);
}

// x^{k+1} = y(lam); the previous iterates shift; partial maxima of |y - x|.
__global__ void __launch_bounds__(MT) k_mma_commit(long long n, double* __restrict__ x,
                                                   double* __restrict__ xo1,
                                                   double* __restrict__ xo2,
                                                   const double* __restrict__ low,
                                                   const double* __restrict__ upp,
                                                   const double* __restrict__ df0,
                                                   const double* __restrict__ df1,
                                                   const unsigned char* __restrict__ active,
                                                   double lam, double xmin, double xmax,
                                                   double move, double scale0, double* partial) {
  double mx = 0.0;
  for (long long j = blockIdx.x * (long long)MT + threadIdx.x; j < n; j += (long long)gridDim.x * MT) {
    const double xj = x[j];
    double y = xj;
    if (!active || active[j])
      y = mma_var(xj, low[j], upp[j], scale0 * df0[j], df1[j], lam, xmin, xmax, move).y;
    xo2[j] = xo1[j];
    xo1[j] = xj;
    x[j] = y;
    mx = fmax(mx, fabs(y - xj));
  }
  block_partial<true>(mx, partial);
}

// out = clamp(in, lo, hi) on active entries, fixed (or 0) elsewhere
__global__ void k_design_map(long long n, const double* in, const unsigned char* __restrict__ active,
                             const double* __restrict__ fixed, double lo, double hi, double* out) {
  const long long j = blockIdx.x * (long long)MT + threadIdx.x;
  if (j >= n) return;
  if (!active || active[j])
    out[j] = fmin(fmax(in[j], lo), hi);
  else
    out[j] = fixed ? fixed[j] : 0.0;
}

inline unsigned grid1(long long n) { return (unsigned)((n + MT - 1) / MT); }

nc_status read_sync(nc_ctx* ctx, const double* d, double* h, int k, cudaStream_t s,
                    const char* what) {
  nc_status st = cuda_check(ctx, cudaMemcpyAsync(h, d, sizeof(double) * k, cudaMemcpyDeviceToHost, s), what);
  if (st != NC_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(s), what);
}

}  // namespace

extern "C" {

void nc_default_mma_opts(nc_mma_opts* o) {
  if (!o) return;
  o->move = 0.2;
  o->xmin = 0.0;
  o->xmax = 1.0;
  o->df0_scale = 1.0;
}

nc_status nc_design_map(nc_ctx* ctx, long long n, const double* in, const unsigned char* active,
                        const double* fixed, double lo, double hi, double* out, void* stream) {
  if (!ctx) return NC_ERR_ARG;
  if (!in || !out || n < 1 || !(hi >= lo))
    return set_err(ctx, NC_ERR_ARG, "nc_design_map: invalid argument");
  k_design_map<<<grid1(n), MT, 0, (cudaStream_t)stream>>>(n, in, active, fixed, lo, hi, out);
  return cuda_check(ctx, cudaGetLastError(), "nc_design_map");
}

nc_status nc_volume(nc_ctx* ctx, long long n, const double* gamma, const unsigned char* active,
                    double vf, double* g_host, double* dgdgamma, void* stream) {
  if (!ctx) return NC_ERR_ARG;
  if (!gamma || !g_host || n < 1 || !(vf > 0.0))
    return set_err(ctx, NC_ERR_ARG, "nc_volume: invalid argument");
  cudaStream_t s = (cudaStream_t)stream;
  k_volume<<<MMA_BLOCKS, MT, 0, s>>>(n, gamma, active, ctx->partial, ctx->partial + MMA_BLOCKS);
  k_fold<<<1, MT, 0, s>>>(MMA_BLOCKS, ctx->partial, ctx->dscal);
  k_fold<<<1, MT, 0, s>>>(MMA_BLOCKS, ctx->partial + MMA_BLOCKS, ctx->dscal + 1);
  double sc[2];
  nc_status st = read_sync(ctx, ctx->dscal, sc, 2, s, "nc_volume");
  if (st != NC_OK) return st;
  if (!(sc[1] > 0.0)) return set_err(ctx, NC_ERR_ARG, "nc_volume: no active variable");
  const double scale = 1.0 / (vf * sc[1]);
  *g_host = sc[0] * scale - 1.0;
  if (dgdgamma) {
    k_volume_grad<<<grid1(n), MT, 0, s>>>(n, active, -scale, dgdgamma);
    return cuda_check(ctx, cudaGetLastError(), "nc_volume gradient");
  }
  return NC_OK;
}

nc_status nc_mma_update(nc_ctx* ctx, long long n, int iter, double* x, double* xold1,
                        double* xold2, double* low, double* upp, const double* df0, double f1,
                        const double* df1, const unsigned char* active, const nc_mma_opts* opts,
                        double* lambda_host, double* change_host, void* stream) {
  if (!ctx) return NC_ERR_ARG;
  nc_mma_opts o;
  nc_default_mma_opts(&o);
  if (opts) o = *opts;
  if (!x || !xold1 || !xold2 || !low || !upp || !df0 || !df1 || n < 1 || iter < 0 ||
      !(o.xmax > o.xmin) || !(o.move > 0.0) || !std::isfinite(f1) || !(o.df0_scale > 0.0))
    return set_err(ctx, NC_ERR_ARG, "nc_mma_update: invalid argument");
  cudaStream_t s = (cudaStream_t)stream;
  k_mma_asym<<<grid1(n), MT, 0, s>>>(n, iter, x, xold1, xold2, low, upp, active, o.xmin, o.xmax);
  nc_status st = NC_OK;
  // approximated constraint at the minimiser of the Lagrangian for lam
  auto g = [&](double lam, double* out) -> nc_status {
    k_mma_dual<<<MMA_BLOCKS, MT, 0, s>>>(n, x, low, upp, df0, df1, active, lam, o.xmin, o.xmax,
                                         o.move, o.df0_scale, ctx->partial);
    k_fold<<<1, MT, 0, s>>>(MMA_BLOCKS, ctx->partial, ctx->dscal);
    double sum;
    nc_status e = read_sync(ctx, ctx->dscal, &sum, 1, s, "nc_mma_update");
    if (e != NC_OK) return e;
    if (!std::isfinite(sum)) return set_err(ctx, NC_ERR_NAN, "nc_mma_update: non-finite value");
    *out = f1 + sum;
    return NC_OK;
  };
  double lam = 0.0, v;
  if ((st = g(0.0, &v)) != NC_OK) return st;
  if (v > 0.0) {
    double hi = 1.0;
    for (int i = 0; i < 200; ++i) {
      if ((st = g(hi, &v)) != NC_OK) return st;
      if (v <= 0.0) break;
      hi *= 2.0;
    }
    double lo = 0.0;
    for (int i = 0; i < 200; ++i) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if ((st = g(mid, &v)) != NC_OK) return st;
      if (v > 0.0)
        lo = mid;
      else
        hi = mid;
    }
    lam = hi;
  }
  k_mma_commit<<<MMA_BLOCKS, MT, 0, s>>>(n, x, xold1, xold2, low, upp, df0, df1, active, lam,
                                         o.xmin, o.xmax, o.move, o.df0_scale, ctx->partial);
  if (lambda_host) *lambda_host = lam;
  std::vector<double> part(MMA_BLOCKS);
  if ((st = read_sync(ctx, ctx->partial, part.data(), MMA_BLOCKS, s, "nc_mma_update")) != NC_OK)
    return st;
  double mx = 0.0;
  for (double p : part) mx = std::fmax(mx, p);
  if (change_host) *change_host = mx;
  return NC_OK;
}

}  // extern "C"
