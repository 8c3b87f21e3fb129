// Direct solve on the coarsest multigrid level.
//
// The coarsest grid is small (e.g. 2^3 or 3^3 elements, a few hundred unknowns),
// so instead of many Krylov iterations -- each a dozen kernel launches on a
// handful of elements -- its Jacobian is formed explicitly and inverted once
// per linearisation:
//   1. a kernel computes every column of every element Jacobian J_e in FP64
//      (the element tangent with unit directions; Dirichlet columns are zero),
//   2. the host assembles the dense matrix (Dirichlet rows identity, Dirichlet
//      columns removed from interior rows, the same operator as nc_jvp) and
//      inverts it by Gauss-Jordan elimination with partial pivoting in FP64,
//   3. the inverse (in the cycle's precision) is applied with one dense
//      matrix-vector kernel: one warp per row, fixed-order shuffle reduction.
#include <cmath>
#include <cstring>
#include <vector>

#include "nc_internal.cuh"

namespace nc {
nc_status set_err(nc_ctx* ctx, nc_status st, const std::string& msg);
nc_status cuda_check(nc_ctx* ctx, cudaError_t e, const char* what);
}  // namespace nc

namespace nc {

namespace {

// One block per element, one thread per column k = f*8 + a of J_e.
template <typename R>
__global__ void k_coarse_elem_jac(LevelDev d, ElemConst<double> c, const R* __restrict__ x,
                                  const R* __restrict__ gam, const R* __restrict__ src,
                                  double* Jel) {
  const long long e = blockIdx.x;
  const int k = threadIdx.x;
  if (k >= 40 || e >= d.E) return;
  int i, j, kk;
  elem_ijk(d, e, i, j, kk);
  const long long sy = d.nx + 1, sz = (long long)(d.nx + 1) * (d.ny + 1);
  const long long n0 = i + sy * (j + (long long)(d.ny + 1) * kk);
  double xe[5][8], ve[5][8], out[5][8];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const long long n = n0 + (a & 1) + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      xe[f][a] = (double)x[f * d.Nn + n];
      ve[f][a] = 0.0;
    }
  }
  const int fk = k / 8, ak = k % 8;
  const long long nk = n0 + (ak & 1) + ((ak >> 1) & 1) * sy + ((ak >> 2) & 1) * sz;
  double* col = Jel + (e * 40 + k) * 40;
  if ((d.flag[nk] >> fk) & 1) {  // Dirichlet column: removed
    for (int r = 0; r < 40; ++r) col[r] = 0.0;
    return;
  }
  ve[fk][ak] = 1.0;
  elem_jvp<double>(xe, ve, (double)gam[e], src ? (double)src[e] : 0.0, c, out);
#pragma unroll
  for (int g = 0; g < 5; ++g)
#pragma unroll
    for (int b = 0; b < 8; ++b) col[g * 8 + b] = out[g][b];
}

// z = A^T b: one thread per column; a warp reads consecutive entries of a row.
template <typename R>
__global__ void k_dense_gemv_t(int n, const R* __restrict__ A, const R* __restrict__ b,
                               R* __restrict__ z) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n) return;
  R acc = R(0);
  for (int i = 0; i < n; ++i) acc += A[(size_t)i * n + col] * b[i];
  z[col] = acc;
}

template <typename R>
__global__ void k_dense_gemv(int n, const R* __restrict__ A, const R* __restrict__ b,
                             R* __restrict__ z) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const R* a = A + (size_t)row * n;
  R acc = R(0);
  for (int j = lane; j < n; j += 32) acc += a[j] * b[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) z[row] = acc;
}

// In-place Gauss-Jordan inverse with partial pivoting (row-major n x n).
// Returns false if a pivot vanishes (the coarse operator is singular).
bool gauss_jordan_inverse(std::vector<double>& A, int n) {
  std::vector<int> perm(n);
  for (int p = 0; p < n; ++p) {
    int q = p;
    double best = std::fabs(A[(size_t)p * n + p]);
    for (int i = p + 1; i < n; ++i) {
      const double v = std::fabs(A[(size_t)i * n + p]);
      if (v > best) { best = v; q = i; }
    }
    perm[p] = q;
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    if (q != p)
      for (int j = 0; j < n; ++j) std::swap(A[(size_t)p * n + j], A[(size_t)q * n + j]);
    double* rp = &A[(size_t)p * n];
    const double inv = 1.0 / rp[p];
    rp[p] = 1.0;
    for (int j = 0; j < n; ++j) rp[j] *= inv;
    for (int i = 0; i < n; ++i) {
      if (i == p) continue;
      double* ri = &A[(size_t)i * n];
      const double f = ri[p];
      if (f == 0.0) continue;
      ri[p] = 0.0;
      for (int j = 0; j < n; ++j) ri[j] -= f * rp[j];
    }
  }
  // undo the row interchanges as column interchanges, in reverse order
  for (int p = n - 1; p >= 0; --p) {
    const int q = perm[p];
    if (q != p)
      for (int i = 0; i < n; ++i) std::swap(A[(size_t)i * n + p], A[(size_t)i * n + q]);
  }
  return true;
}

}  // namespace

int coarse_dense_dofs(const Level& L) { return (int)(5 * L.d.Nn); }

template <typename R>
nc_status coarse_setup(nc_ctx* ctx, Level& L, const R* x, const R* gam, const R* src,
                       R** inv_dev, cudaStream_t s) {
  const int n = coarse_dense_dofs(L);
  const long long E = L.d.E;
  nc_status st;
  if (ctx->cjel_elems < E) {
    cudaFree(ctx->cjel);
    ctx->cjel = nullptr;
    ctx->cjel_elems = 0;
    if ((st = cuda_check(ctx, cudaMalloc((void**)&ctx->cjel, sizeof(double) * 1600 * E),
                         "cudaMalloc coarse")) != NC_OK)
      return st;
    ctx->cjel_elems = E;
  }
  if (!*inv_dev) {
    if ((st = cuda_check(ctx, cudaMalloc((void**)inv_dev, sizeof(R) * (size_t)n * n),
                         "cudaMalloc coarse inverse")) != NC_OK)
      return st;
  }
  k_coarse_elem_jac<R><<<(unsigned)E, 64, 0, s>>>(L.d, L.c64, x, gam, src, ctx->cjel);
  std::vector<double> jel((size_t)1600 * E);
  std::vector<uint8_t> fl((size_t)L.d.Nn);
  if ((st = cuda_check(ctx, cudaMemcpyAsync(jel.data(), ctx->cjel, sizeof(double) * jel.size(),
                                            cudaMemcpyDeviceToHost, s), "coarse D2H")) != NC_OK ||
      (st = cuda_check(ctx, cudaMemcpyAsync(fl.data(), L.flag, fl.size(), cudaMemcpyDeviceToHost, s),
                       "coarse flags D2H")) != NC_OK ||
      (st = cuda_check(ctx, cudaStreamSynchronize(s), "coarse sync")) != NC_OK)
    return st;
  // dense assembly, unknown index f * Nn + node
  const LevelDev& d = L.d;
  const long long Nn = d.Nn;
  std::vector<double> A((size_t)n * n, 0.0);
  const long long sy = d.nx + 1, sz = (long long)(d.nx + 1) * (d.ny + 1);
  for (long long e = 0; e < E; ++e) {
    int i, j, kk;
    elem_ijk(d, e, i, j, kk);
    const long long n0 = i + sy * (j + (long long)(d.ny + 1) * kk);
    long long nodes[8];
    for (int a = 0; a < 8; ++a) nodes[a] = n0 + (a & 1) + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz;
    for (int k = 0; k < 40; ++k) {
      const long long col = (k / 8) * Nn + nodes[k % 8];
      const double* cj = &jel[(size_t)(e * 40 + k) * 40];
      for (int r = 0; r < 40; ++r) {
        const long long row = (r / 8) * Nn + nodes[r % 8];
        A[(size_t)row * n + col] += cj[r];
      }
    }
  }
  for (long long node = 0; node < Nn; ++node)
    for (int f = 0; f < 5; ++f)
      if ((fl[node] >> f) & 1) {
        const long long r = f * Nn + node;
        for (int c = 0; c < n; ++c) A[(size_t)r * n + c] = 0.0;
        A[(size_t)r * n + r] = 1.0;
      }
  if (!gauss_jordan_inverse(A, n))
    return set_err(ctx, NC_ERR_NAN, "coarsest-level operator is singular");
  std::vector<R> Ar(A.begin(), A.end());
  if ((st = cuda_check(ctx, cudaMemcpyAsync(*inv_dev, Ar.data(), sizeof(R) * Ar.size(),
                                            cudaMemcpyHostToDevice, s), "coarse H2D")) != NC_OK)
    return st;
  return cuda_check(ctx, cudaStreamSynchronize(s), "coarse sync");
}

template <typename R>
nc_status coarse_setup_stencil(nc_ctx* ctx, Level& L, const R* S, R** inv_dev, cudaStream_t s) {
  const int n = coarse_dense_dofs(L);
  const LevelDev& d = L.d;
  const long long Nn = d.Nn;
  nc_status st;
  if (!*inv_dev) {
    if ((st = cuda_check(ctx, cudaMalloc((void**)inv_dev, sizeof(R) * (size_t)n * n),
                         "cudaMalloc coarse inverse")) != NC_OK)
      return st;
  }
  std::vector<R> sh((size_t)STENCIL_VALUES * Nn);
  if ((st = cuda_check(ctx, cudaMemcpyAsync(sh.data(), S, sizeof(R) * sh.size(),
                                            cudaMemcpyDeviceToHost, s), "coarse stencil D2H")) != NC_OK ||
      (st = cuda_check(ctx, cudaStreamSynchronize(s), "coarse sync")) != NC_OK)
    return st;
  // dense assembly, unknown index f * Nn + node; Dirichlet rows are identity rows
  // of the stencil already
  std::vector<double> A((size_t)n * n, 0.0);
  for (long long node = 0; node < Nn; ++node) {
    int i, j, k;
    node_ijk(d, node, i, j, k);
    for (int o = 0; o < 27; ++o) {
      const int ii = i + o % 3 - 1, jj = j + (o / 3) % 3 - 1, kk = k + o / 9 - 1;
      if (ii < 0 || ii > d.nx || jj < 0 || jj > d.ny || kk < 0 || kk > d.nz) continue;
      const long long m = ii + (long long)(d.nx + 1) * (jj + (long long)(d.ny + 1) * kk);
      for (int f = 0; f < 5; ++f)
        for (int g = 0; g < 5; ++g)
          A[(size_t)(f * Nn + node) * n + (g * Nn + m)] =
              (double)sh[(size_t)((o * 5 + f) * 5 + g) * Nn + node];
    }
  }
  if (!gauss_jordan_inverse(A, n))
    return set_err(ctx, NC_ERR_NAN, "coarsest-level Galerkin operator is singular");
  std::vector<R> Ar(A.begin(), A.end());
  if ((st = cuda_check(ctx, cudaMemcpyAsync(*inv_dev, Ar.data(), sizeof(R) * Ar.size(),
                                            cudaMemcpyHostToDevice, s), "coarse H2D")) != NC_OK)
    return st;
  return cuda_check(ctx, cudaStreamSynchronize(s), "coarse sync");
}

template <typename R>
void coarse_apply(const Level& L, bool tr, const R* inv, const R* b, R* z, cudaStream_t s) {
  const int n = coarse_dense_dofs(L);
  if (tr)
    k_dense_gemv_t<R><<<(n + 127) / 128, 128, 0, s>>>(n, inv, b, z);
  else
    k_dense_gemv<R><<<(n + 7) / 8, 256, 0, s>>>(n, inv, b, z);
}

template nc_status coarse_setup<double>(nc_ctx*, Level&, const double*, const double*,
                                        const double*, double**, cudaStream_t);
template nc_status coarse_setup<float>(nc_ctx*, Level&, const float*, const float*, const float*,
                                       float**, cudaStream_t);
template void coarse_apply<double>(const Level&, bool, const double*, const double*, double*,
                                   cudaStream_t);
template nc_status coarse_setup_stencil<double>(nc_ctx*, Level&, const double*, double**,
                                                cudaStream_t);
template nc_status coarse_setup_stencil<float>(nc_ctx*, Level&, const float*, float**,
                                               cudaStream_t);
template void coarse_apply<float>(const Level&, bool, const float*, const float*, float*,
                                  cudaStream_t);

}  // namespace nc
