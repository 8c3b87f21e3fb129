// Vector kernels: casts, axpy variants and deterministic reductions.
//
// Reductions use a fixed partition that depends only on the vector length:
// each block folds a grid-stride range into one partial with a warp-shuffle
// tree, and a second single-block kernel folds the partials in index order.
// Results are bitwise reproducible from run to run.
#include "nc_internal.cuh"

namespace nc {

namespace {

constexpr int VT = 256;

inline unsigned vblocks(long long n) {
  long long b = (n + VT * 4 - 1) / (VT * 4);
  if (b < 1) b = 1;
  if (b > 4 * RED_BLOCKS_MAX) b = 4 * RED_BLOCKS_MAX;
  return (unsigned)b;
}

inline int red_blocks(long long n) {
  long long b = (n + RED_THREADS * 8 - 1) / (RED_THREADS * 8);
  if (b < 1) b = 1;
  if (b > RED_BLOCKS_MAX) b = RED_BLOCKS_MAX;
  return (int)b;
}

template <typename Rd, typename Rs>
__global__ void k_cast(long long n, const Rs* __restrict__ x, Rd* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = Rd(x[i]);
}

template <typename R>
__global__ void k_axpy(long long n, R a, const R* __restrict__ x, R* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

template <typename R>
__global__ void k_xpay(long long n, const R* __restrict__ x, R a, R* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] + a * y[i];
}

template <typename R>
__global__ void k_waxpy(long long n, const R* __restrict__ x, R a, const R* __restrict__ y,
                        R* __restrict__ w) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    w[i] = x[i] + a * y[i];
}

template <typename R>
__global__ void k_div(long long n, const R* __restrict__ x, const R* __restrict__ d,
                      R* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i] / d[i];
}

template <typename R>
__global__ void k_scal(long long n, R a, R* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] *= a;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-level sum of one value per thread, result valid in thread 0.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T r = T(0);
  if (wid == 0) {
    r = lane < (int)(blockDim.x >> 5) ? sh[lane] : T(0);
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

// partial[i * nb + b] = sum over block b's range of X_i . y  (accumulated in R)
template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_mdot_partial(long long n, int k,
                                                              const R* __restrict__ X, long long ld,
                                                              const R* __restrict__ y,
                                                              double* partial) {
  __shared__ R sh[RED_THREADS / 32];
  const int nb = gridDim.x;
  const long long stride = (long long)nb * blockDim.x;
  const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  constexpr int KB = 4;  // vectors per pass
  for (int i = 0; i < k; i += KB) {
    R acc[KB] = {R(0), R(0), R(0), R(0)};
    for (long long t = i0; t < n; t += stride) {
      const R yt = y[t];
#pragma unroll
      for (int q = 0; q < KB; ++q)
        if (i + q < k) acc[q] += X[(i + q) * ld + t] * yt;
    }
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      if (i + q >= k) break;
      const R s = block_sum(acc[q], sh);
      if (threadIdx.x == 0) partial[(i + q) * nb + blockIdx.x] = double(s);
    }
  }
}

__global__ void __launch_bounds__(RED_THREADS) k_mdot_final(int nb, const double* partial,
                                                            double* out, int take_sqrt) {
  __shared__ double sh[RED_THREADS / 32];
  const int i = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += partial[i * nb + b];
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) out[i] = take_sqrt ? sqrt(fmax(s, 0.0)) : s;
}

// y -= sum_i coef[i] X_i, and partial[b] = sum of y^2 over block b's range
template <typename R>
__global__ void __launch_bounds__(RED_THREADS) k_maxpy_norm(long long n, int k,
                                                            const R* __restrict__ X, long long ld,
                                                            const double* __restrict__ coef,
                                                            R* __restrict__ y, double* partial) {
  __shared__ R c[MAX_RESTART + 1];
  __shared__ R sh[RED_THREADS / 32];
  for (int i = threadIdx.x; i < k; i += blockDim.x) c[i] = R(coef[i]);
  __syncthreads();
  R acc2 = R(0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    R acc = y[t];
    for (int i = 0; i < k; ++i) acc -= c[i] * X[i * ld + t];
    y[t] = acc;
    acc2 += acc * acc;
  }
  const R s = block_sum(acc2, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = double(s);
}

// v = x / *nrm (zero on a vanishing or non-finite norm) and t = v / d
template <typename R>
__global__ void k_scale_div(long long n, const R* __restrict__ x, const double* __restrict__ nrm,
                            const R* __restrict__ d, R* __restrict__ v, R* __restrict__ t) {
  const double nv = *nrm;
  const R s = (nv > 0.0 && nv < 1e300) ? R(1.0 / nv) : R(0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const R a = x[i] * s;
    v[i] = a;
    t[i] = a / d[i];
  }
}

// z (+)= (sum_i y[i] X_i) / d
template <typename R>
__global__ void k_combine_div(long long n, int k, const R* __restrict__ X, long long ld,
                              const double* __restrict__ y, const R* __restrict__ d, R* z,
                              int accumulate) {
  __shared__ R c[MAX_RESTART + 1];
  for (int i = threadIdx.x; i < k; i += blockDim.x) c[i] = R(y[i]);
  __syncthreads();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    R acc = R(0);
    for (int i = 0; i < k; ++i) acc += c[i] * X[i * ld + t];
    acc /= d[t];
    z[t] = accumulate ? z[t] + acc : acc;
  }
}

template <typename R>
__global__ void k_maxpy(long long n, int k, const R* __restrict__ X, long long ld,
                        const double* __restrict__ coef, double sign, R* __restrict__ y) {
  __shared__ R c[MAX_RESTART + 1];
  for (int i = threadIdx.x; i < k; i += blockDim.x) c[i] = R(sign * coef[i]);
  __syncthreads();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    R acc = y[t];
    for (int i = 0; i < k; ++i) acc -= c[i] * X[i * ld + t];
    y[t] = acc;
  }
}

// y = x / nrm, with nrm a device scalar; a zero or non-finite norm gives y = 0
// (the Krylov space is exhausted: the caller's least-squares solve handles it).
template <typename R>
__global__ void k_scale_inv(long long n, const R* __restrict__ x, const double* __restrict__ nrm,
                            R* __restrict__ y) {
  const double v = *nrm;
  const R s = (v > 0.0 && v < 1e300) ? R(1.0 / v) : R(0);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x)
    y[t] = x[t] * s;
}

__global__ void k_sqrt_store(const double* in, double* out) { *out = sqrt(fmax(*in, 0.0)); }

}  // namespace

template <typename Rd, typename Rs>
void vcast(long long n, const Rs* x, Rd* y, cudaStream_t s) {
  k_cast<Rd, Rs><<<vblocks(n), VT, 0, s>>>(n, x, y);
}
template <typename R>
void vcopy(long long n, const R* x, R* y, cudaStream_t s) {
  cudaMemcpyAsync(y, x, sizeof(R) * n, cudaMemcpyDeviceToDevice, s);
}
template <typename R>
void vzero(long long n, R* x, cudaStream_t s) {
  cudaMemsetAsync(x, 0, sizeof(R) * n, s);
}
template <typename R>
void vaxpy(long long n, R a, const R* x, R* y, cudaStream_t s) {
  k_axpy<R><<<vblocks(n), VT, 0, s>>>(n, a, x, y);
}
template <typename R>
void vxpay(long long n, const R* x, R a, R* y, cudaStream_t s) {
  k_xpay<R><<<vblocks(n), VT, 0, s>>>(n, x, a, y);
}
template <typename R>
void vwaxpy(long long n, const R* x, R a, const R* y, R* w, cudaStream_t s) {
  k_waxpy<R><<<vblocks(n), VT, 0, s>>>(n, x, a, y, w);
}
template <typename R>
void vdiv(long long n, const R* x, const R* d, R* y, cudaStream_t s) {
  k_div<R><<<vblocks(n), VT, 0, s>>>(n, x, d, y);
}
template <typename R>
void vscal(long long n, R a, R* y, cudaStream_t s) {
  k_scal<R><<<vblocks(n), VT, 0, s>>>(n, a, y);
}
template <typename R>
void vmdot(long long n, int k, const R* X, long long ld, const R* y, double* out, double* partial,
           cudaStream_t s) {
  const int nb = red_blocks(n);
  k_mdot_partial<R><<<nb, RED_THREADS, 0, s>>>(n, k, X, ld, y, partial);
  k_mdot_final<<<k, RED_THREADS, 0, s>>>(nb, partial, out, 0);
}
template <typename R>
void vnorm(long long n, const R* x, double* out, double* partial, cudaStream_t s) {
  const int nb = red_blocks(n);
  k_mdot_partial<R><<<nb, RED_THREADS, 0, s>>>(n, 1, x, 0, x, partial);
  k_mdot_final<<<1, RED_THREADS, 0, s>>>(nb, partial, out, 1);
}
template <typename R>
void vmaxpy_norm(long long n, int k, const R* X, long long ld, const double* coef, R* y,
                 double* out_norm, double* partial, cudaStream_t s) {
  const int nb = red_blocks(n);
  k_maxpy_norm<R><<<nb, RED_THREADS, 0, s>>>(n, k, X, ld, coef, y, partial);
  k_mdot_final<<<1, RED_THREADS, 0, s>>>(nb, partial, out_norm, 1);
}
template <typename R>
void vscale_div(long long n, const R* x, const double* nrm, const R* d, R* v, R* t,
                cudaStream_t s) {
  k_scale_div<R><<<vblocks(n), VT, 0, s>>>(n, x, nrm, d, v, t);
}
template <typename R>
void vcombine_div(long long n, int k, const R* X, long long ld, const double* y, const R* d, R* z,
                  bool accumulate, cudaStream_t s) {
  k_combine_div<R><<<vblocks(n), VT, 0, s>>>(n, k, X, ld, y, d, z, accumulate ? 1 : 0);
}
template <typename R>
void vmaxpy(long long n, int k, const R* X, long long ld, const double* coef, double sign, R* y,
            cudaStream_t s) {
  k_maxpy<R><<<vblocks(n), VT, 0, s>>>(n, k, X, ld, coef, sign, y);
}
template <typename R>
void vscale_inv(long long n, const R* x, const double* nrm, R* y, cudaStream_t s) {
  k_scale_inv<R><<<vblocks(n), VT, 0, s>>>(n, x, nrm, y);
}
void dev_sqrt_store(const double* in, double* out, cudaStream_t s) {
  k_sqrt_store<<<1, 1, 0, s>>>(in, out);
}

template void vcast<float, double>(long long, const double*, float*, cudaStream_t);
template void vcast<double, float>(long long, const float*, double*, cudaStream_t);
#define NC_INST(R)                                                                             \
  template void vcopy<R>(long long, const R*, R*, cudaStream_t);                               \
  template void vzero<R>(long long, R*, cudaStream_t);                                         \
  template void vaxpy<R>(long long, R, const R*, R*, cudaStream_t);                            \
  template void vxpay<R>(long long, const R*, R, R*, cudaStream_t);                            \
  template void vwaxpy<R>(long long, const R*, R, const R*, R*, cudaStream_t);                 \
  template void vdiv<R>(long long, const R*, const R*, R*, cudaStream_t);                      \
  template void vscal<R>(long long, R, R*, cudaStream_t);                                      \
  template void vmdot<R>(long long, int, const R*, long long, const R*, double*, double*,      \
                         cudaStream_t);                                                        \
  template void vmaxpy<R>(long long, int, const R*, long long, const double*, double, R*,      \
                          cudaStream_t);                                                       \
  template void vscale_inv<R>(long long, const R*, const double*, R*, cudaStream_t);            \
  template void vnorm<R>(long long, const R*, double*, double*, cudaStream_t);                 \
  template void vmaxpy_norm<R>(long long, int, const R*, long long, const double*, R*, double*, \
                               double*, cudaStream_t);                                         \
  template void vscale_div<R>(long long, const R*, const double*, const R*, R*, R*,           \
                              cudaStream_t);                                                   \
  template void vcombine_div<R>(long long, int, const R*, long long, const double*, const R*,  \
                                R*, bool, cudaStream_t);
NC_INST(double)
NC_INST(float)
#undef NC_INST

}  // namespace nc
