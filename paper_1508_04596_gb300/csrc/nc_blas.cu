// Vector kernels: casts, axpy variants, deterministic reductions and the fused
// Gram-Schmidt / Arnoldi passes of the Krylov solvers.
//
// Every kernel is HBM-bound: it walks its vectors in chunks of four elements,
// moved as 16-byte packets (float4- / 2 x double2-wide) when every pointer it
// touches is 16-byte aligned, and element by element otherwise; the n mod 4
// tail is taken by the first threads.  Multivectors are stored with a padded
// leading dimension (a multiple of 64 elements) so that every column is aligned.
//
// Reductions use a fixed partition that depends only on the vector length:
// each block folds a grid-stride range of chunks into one partial with a
// warp-shuffle tree, and a second single-block kernel folds the partials in
// index order.  Results are bitwise reproducible from run to run.
#include <cstdint>

#include "nc_internal.cuh"

namespace nc {

namespace {

constexpr int VT = 256;
constexpr int MAP_BLOCKS_MAX = 8 * 152;  // streaming kernels: one wave of 256-thread blocks

template <typename R>
struct __align__(16) P4 {
  R v[4];
};

inline bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline unsigned map_blocks(long long n) {
  long long b = (n / 4 + VT - 1) / VT;
  if (b < 1) b = 1;
  if (b > MAP_BLOCKS_MAX) b = MAP_BLOCKS_MAX;
  return (unsigned)b;
}

inline int red_blocks(long long n) {
  long long b = (n + RED_THREADS * 8 - 1) / (RED_THREADS * 8);
  if (b < 1) b = 1;
  if (b > RED_BLOCKS_MAX) b = RED_BLOCKS_MAX;
  return (int)b;
}

template <typename R, bool VEC>
__device__ __forceinline__ void ld4(const R* __restrict__ p, long long c, R o[4]) {
  if (VEC) {
    const P4<R> t = reinterpret_cast<const P4<R>*>(p)[c];
#pragma unroll
    for (int u = 0; u < 4; ++u) o[u] = t.v[u];
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) o[u] = p[4 * c + u];
  }
}

template <typename R, bool VEC>
__device__ __forceinline__ void st4(R* __restrict__ p, long long c, const R o[4]) {
  if (VEC) {
    P4<R> t;
#pragma unroll
    for (int u = 0; u < 4; ++u) t.v[u] = o[u];
    reinterpret_cast<P4<R>*>(p)[c] = t;
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) p[4 * c + u] = o[u];
  }
}

// Chunk loop of a streaming kernel: chunks c < n/4 by grid stride (f4), then
// the tail element n4*4 + gid for gid < n mod 4 (f1).
template <typename F4, typename F1>
__device__ __forceinline__ void chunk_loop(long long n, F4&& f4, F1&& f1) {
  const long long n4 = n >> 2;
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)gridDim.x * blockDim.x;
  for (long long c = gid; c < n4; c += gs) f4(c);
  if (gid < (n & 3)) f1(n4 * 4 + gid);
}

template <typename Rd, typename Rs, bool VEC>
__global__ void k_cast(long long n, const Rs* __restrict__ x, Rd* __restrict__ y) {
  chunk_loop(n, [&](long long c) {
    Rs a[4];
    Rd b[4];
    ld4<Rs, VEC>(x, c, a);
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = Rd(a[u]);
    st4<Rd, VEC>(y, c, b);
  }, [&](long long i) { y[i] = Rd(x[i]); });
}

template <typename R, bool VEC>
__global__ void k_axpy(long long n, R a, const R* __restrict__ x, R* __restrict__ y) {
  chunk_loop(n, [&](long long c) {
    R xv[4], yv[4];
    ld4<R, VEC>(x, c, xv);
    ld4<R, VEC>(y, c, yv);
#pragma unroll
    for (int u = 0; u < 4; ++u) yv[u] += a * xv[u];
    st4<R, VEC>(y, c, yv);
  }, [&](long long i) { y[i] += a * x[i]; });
}

template <typename R, bool VEC>
__global__ void k_xpay(long long n, const R* __restrict__ x, R a, R* __restrict__ y) {
  chunk_loop(n, [&](long long c) {
    R xv[4], yv[4];
    ld4<R, VEC>(x, c, xv);
    ld4<R, VEC>(y, c, yv);
#pragma unroll
    for (int u = 0; u < 4; ++u) yv[u] = xv[u] + a * yv[u];
    st4<R, VEC>(y, c, yv);
  }, [&](long long i) { y[i] = x[i] + a * y[i]; });
}

template <typename R, bool VEC>
__global__ void k_waxpy(long long n, const R* __restrict__ x, R a, const R* __restrict__ y,
                        R* __restrict__ w) {
  chunk_loop(n, [&](long long c) {
    R xv[4], yv[4];
    ld4<R, VEC>(x, c, xv);
    ld4<R, VEC>(y, c, yv);
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] += a * yv[u];
    st4<R, VEC>(w, c, xv);
  }, [&](long long i) { w[i] = x[i] + a * y[i]; });
}

template <typename R, bool VEC>
__global__ void k_div(long long n, const R* __restrict__ x, const R* __restrict__ d,
                      R* __restrict__ y) {
  chunk_loop(n, [&](long long c) {
    R xv[4], dv[4];
    ld4<R, VEC>(x, c, xv);
    ld4<R, VEC>(d, c, dv);
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] /= dv[u];
    st4<R, VEC>(y, c, xv);
  }, [&](long long i) { y[i] = x[i] / d[i]; });
}

template <typename R, bool VEC>
__global__ void k_scal(long long n, R a, R* __restrict__ y) {
  chunk_loop(n, [&](long long c) {
    R yv[4];
    ld4<R, VEC>(y, c, yv);
#pragma unroll
    for (int u = 0; u < 4; ++u) yv[u] *= a;
    st4<R, VEC>(y, c, yv);
  }, [&](long long i) { y[i] *= a; });
}

// y = x / nrm, with nrm a device scalar; a zero or non-finite norm gives y = 0
// (the Krylov space is exhausted: the caller's least-squares solve handles it).
template <typename R, bool VEC>
__global__ void k_scale_inv(long long n, const R* __restrict__ x, const double* __restrict__ nrm,
                            R* __restrict__ y) {
  __shared__ R s_sh;
  if (threadIdx.x == 0) {
    const double v = *nrm;
    s_sh = (v > 0.0 && v < 1e300) ? R(1.0 / v) : R(0);
  }
  __syncthreads();
  const R s = s_sh;
  chunk_loop(n, [&](long long c) {
    R xv[4];
    ld4<R, VEC>(x, c, xv);
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] *= s;
    st4<R, VEC>(y, c, xv);
  }, [&](long long i) { y[i] = x[i] * s; });
}

// a[u] -= sum_{q < k} cf[q] X_q[chunk c][u], four columns per round so that four
// packet loads per thread are in flight.
template <typename R, bool VEC>
__device__ __forceinline__ void sub_cols(const R* __restrict__ X, long long ld, int k, const R* cf,
                                         long long c, R a[4]) {
  int q = 0;
  for (; q + 4 <= k; q += 4) {
    R xv[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r) ld4<R, VEC>(X + (q + r) * ld, c, xv[r]);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] -= cf[q + r] * xv[r][u];
  }
  for (; q < k; ++q) {
    R xv[4];
    ld4<R, VEC>(X + q * ld, c, xv);
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] -= cf[q] * xv[u];
  }
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

// partial[i * nb + b] = sum over block b's chunks of X_i . y for i < k, and with
// self also partial[k * nb + b] = y . y  (per-thread sums in R, partials in double)
template <typename R, bool VEC>
__global__ void __launch_bounds__(RED_THREADS) k_mdot_partial(long long n, int k,
                                                              const R* __restrict__ X, long long ld,
                                                              const R* __restrict__ y, int self,
                                                              double* partial) {
  __shared__ R sh[RED_THREADS / 32];
  constexpr int KB = sizeof(R) == 8 ? 4 : 8;  // columns per pass over y (FP64: fewer live loads)
  const int nb = gridDim.x;
  const long long n4 = n >> 2;
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long gs = (long long)nb * blockDim.x;
  const int passes = k > 0 ? (k + KB - 1) / KB : 1;
  for (int p = 0; p < passes; ++p) {
    const int i0 = p * KB;
    const bool do_self = self && p == 0;
    // FP32 (HBM-bound): two chunks per iteration and two accumulators per column
    // keep more loads in flight and shorten the FMA chains.  FP64 runs at 1/64 of
    // the FP32 rate on this GPU, so an FP64 multi-dot is bound by its FMA count:
    // one FMA per element, one chunk per iteration.
    constexpr int CU = sizeof(R) == 4 ? 2 : 1;
    R acc[KB], acc2[KB], accs = R(0);
#pragma unroll
    for (int q = 0; q < KB; ++q) acc[q] = acc2[q] = R(0);
    for (long long c0 = gid; c0 < n4; c0 += CU * gs) {
#pragma unroll
      for (int h = 0; h < CU; ++h) {
        const long long c = c0 + h * gs;
        if (c >= n4) break;
        R yv[4];
        ld4<R, VEC>(y, c, yv);
        if (do_self) {
#pragma unroll
          for (int u = 0; u < 4; ++u) accs = fma(yv[u], yv[u], accs);
        }
#pragma unroll
        for (int q = 0; q < KB; ++q) {
          if (i0 + q < k) {
            R xv[4];
            ld4<R, VEC>(X + (i0 + q) * ld, c, xv);
            if (CU == 2) {
              acc[q] = fma(xv[0], yv[0], acc[q]);
              acc2[q] = fma(xv[1], yv[1], acc2[q]);
              acc[q] = fma(xv[2], yv[2], acc[q]);
              acc2[q] = fma(xv[3], yv[3], acc2[q]);
            } else {
#pragma unroll
              for (int u = 0; u < 4; ++u) acc[q] = fma(xv[u], yv[u], acc[q]);
            }
          }
        }
      }
    }
    if (gid < (n & 3)) {
      const long long i = n4 * 4 + gid;
      const R yt = y[i];
      if (do_self) accs += yt * yt;
#pragma unroll
      for (int q = 0; q < KB; ++q)
        if (i0 + q < k) acc[q] += X[(i0 + q) * ld + i] * yt;
    }
#pragma unroll
    for (int q = 0; q < KB; ++q) {
      if (i0 + q >= k) break;
      const R s = block_sum(acc[q] + acc2[q], sh);
      if (threadIdx.x == 0) partial[(i0 + q) * nb + blockIdx.x] = double(s);
    }
    if (do_self) {
      const R s = block_sum(accs, sh);
      if (threadIdx.x == 0) partial[k * nb + blockIdx.x] = double(s);
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

// One Arnoldi step of the smoother with an unnormalised basis.  With the dots
// g_i = v_i . w (i < k) and the squared basis norms sig2_i:
//   w <- (w - sum_i (g_i / sig2_i) v_i) / sqrt(sig2_{k-1}),   t = w / D (if t),
// and partial[b] = block b's share of ||w||^2 (the next sig2).
template <typename R, bool VEC>
__global__ void __launch_bounds__(RED_THREADS) k_arnoldi_update(long long n, int k,
                                                                const R* __restrict__ X, long long ld,
                                                                const double* __restrict__ g,
                                                                const double* __restrict__ sig2,
                                                                const R* __restrict__ D,
                                                                R* __restrict__ w, R* __restrict__ t,
                                                                double* partial) {
  __shared__ R cf[MAX_RESTART + 1];
  __shared__ R sh[RED_THREADS / 32];
  __shared__ R sc_sh;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const double s2 = sig2[i];
    cf[i] = (s2 > 0.0 && s2 < 1e300) ? R(g[i] / s2) : R(0);
  }
  if (threadIdx.x == 0) {  // FP64 scalar work once per block
    const double sl = sig2[k - 1];
    sc_sh = (sl > 0.0 && sl < 1e300) ? R(1.0 / sqrt(sl)) : R(0);
  }
  __syncthreads();
  const R sc = sc_sh;
  R acc2 = R(0);
  chunk_loop(n, [&](long long c) {
    R a[4];
    ld4<R, VEC>(w, c, a);
    sub_cols<R, VEC>(X, ld, k, cf, c, a);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a[u] *= sc;
      acc2 += a[u] * a[u];
    }
    st4<R, VEC>(w, c, a);
    if (t) {
      R dv[4];
      ld4<R, VEC>(D, c, dv);
#pragma unroll
      for (int u = 0; u < 4; ++u) dv[u] = a[u] / dv[u];
      st4<R, VEC>(t, c, dv);
    }
  }, [&](long long i) {
    R a = w[i];
    for (int q = 0; q < k; ++q) a -= cf[q] * X[q * ld + i];
    a *= sc;
    acc2 += a * a;
    w[i] = a;
    if (t) t[i] = a / D[i];
  });
  const R s = block_sum(acc2, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = double(s);
}

// First basis vector of the smoother: v0 = r (copied unless r is v0 itself),
// t = r / D, partial[b] = block b's share of ||r||^2.
template <typename R, bool VEC>
__global__ void __launch_bounds__(RED_THREADS) k_init_basis(long long n, const R* r,
                                                            const R* __restrict__ D, R* v0,
                                                            R* __restrict__ t, double* partial) {
  __shared__ R sh[RED_THREADS / 32];
  const bool copy = r != v0;
  R acc2 = R(0);
  chunk_loop(n, [&](long long c) {
    R a[4], dv[4];
    ld4<R, VEC>(r, c, a);
    ld4<R, VEC>(D, c, dv);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc2 += a[u] * a[u];
      dv[u] = a[u] / dv[u];
    }
    if (copy) st4<R, VEC>(v0, c, a);
    st4<R, VEC>(t, c, dv);
  }, [&](long long i) {
    const R a = r[i];
    acc2 += a * a;
    if (copy) v0[i] = a;
    t[i] = a / D[i];
  });
  const R s = block_sum(acc2, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = double(s);
}

// z (+)= (sum_i coef[i] X_i) / D   (no division when D is null)
template <typename R, bool VEC>
__global__ void k_combine(long long n, int k, const R* __restrict__ X, long long ld,
                          const double* __restrict__ coef, const R* __restrict__ D, R* z,
                          int accumulate) {
  __shared__ R cf[MAX_RESTART + 1];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cf[i] = R(-coef[i]);
  __syncthreads();
  chunk_loop(n, [&](long long c) {
    R a[4] = {R(0), R(0), R(0), R(0)};
    sub_cols<R, VEC>(X, ld, k, cf, c, a);  // cf holds the negated coefficients
    if (D) {
      R dv[4];
      ld4<R, VEC>(D, c, dv);
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] /= dv[u];
    }
    if (accumulate) {
      R zv[4];
      ld4<R, VEC>(z, c, zv);
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] += zv[u];
    }
    st4<R, VEC>(z, c, a);
  }, [&](long long i) {
    R a = R(0);
    for (int q = 0; q < k; ++q) a -= cf[q] * X[q * ld + i];
    if (D) a /= D[i];
    z[i] = accumulate ? z[i] + a : a;
  });
}

// y -= sign * sum_i coef[i] X_i
template <typename R, bool VEC>
__global__ void k_maxpy(long long n, int k, const R* __restrict__ X, long long ld,
                        const double* __restrict__ coef, double sign, R* __restrict__ y) {
  __shared__ R cf[MAX_RESTART + 1];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cf[i] = R(sign * coef[i]);
  __syncthreads();
  chunk_loop(n, [&](long long c) {
    R a[4];
    ld4<R, VEC>(y, c, a);
    sub_cols<R, VEC>(X, ld, k, cf, c, a);
    st4<R, VEC>(y, c, a);
  }, [&](long long i) {
    R a = y[i];
    for (int q = 0; q < k; ++q) a -= cf[q] * X[q * ld + i];
    y[i] = a;
  });
}

// y -= sign * sum_i coef[i] X_i with FP32 columns and an FP64 y (FP64 arithmetic,
// the same order of operations as k_maxpy<double> on the cast columns)
template <bool VEC>
__global__ void k_maxpy_f32x(long long n, int k, const float* __restrict__ X, long long ld,
                             const double* __restrict__ coef, double sign,
                             double* __restrict__ y) {
  __shared__ double cf[MAX_RESTART + 1];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cf[i] = sign * coef[i];
  __syncthreads();
  chunk_loop(n, [&](long long c) {
    double a[4];
    ld4<double, VEC>(y, c, a);
    int q = 0;
    for (; q + 4 <= k; q += 4) {
      float xv[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r) ld4<float, VEC>(X + (q + r) * ld, c, xv[r]);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] -= cf[q + r] * (double)xv[r][u];
    }
    for (; q < k; ++q) {
      float xv[4];
      ld4<float, VEC>(X + q * ld, c, xv);
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] -= cf[q] * (double)xv[u];
    }
    st4<double, VEC>(y, c, a);
  }, [&](long long i) {
    double a = y[i];
    for (int q = 0; q < k; ++q) a -= cf[q] * (double)X[q * ld + i];
    y[i] = a;
  });
}

// Second classical Gram-Schmidt pass with the normalisation folded in:
// y <- (y - sum_i h_i X_i) / nw,  nw = sqrt(q - sum_i h_i^2)  with q = ||y||^2 on
// entry (h and q from one fused multi-dot; X orthonormal, so nw is the norm of
// the corrected y).  nw is written to *nw_out; a vanishing nw leaves the
// vector unscaled (the caller sees nw = 0 and stops).
template <typename R, bool VEC>
__global__ void k_maxpy_scale(long long n, int k, const R* __restrict__ X, long long ld,
                              const double* __restrict__ h, const double* __restrict__ q,
                              double* nw_out, R* __restrict__ y) {
  __shared__ R cf[MAX_RESTART + 1];
  __shared__ R sc_sh;
  for (int i = threadIdx.x; i < k; i += blockDim.x) cf[i] = R(h[i]);
  if (threadIdx.x == 0) {  // FP64 scalar work once per block
    double hh = 0.0;
    for (int i = 0; i < k; ++i) hh += h[i] * h[i];
    const double nw2 = *q - hh;
    const double nw = nw2 > 0.0 ? sqrt(nw2) : 0.0;
    sc_sh = (nw > 0.0 && nw < 1e300) ? R(1.0 / nw) : R(1);
    if (blockIdx.x == 0) *nw_out = nw;
  }
  __syncthreads();
  const R sc = sc_sh;
  chunk_loop(n, [&](long long c) {
    R a[4];
    ld4<R, VEC>(y, c, a);
    sub_cols<R, VEC>(X, ld, k, cf, c, a);
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] *= sc;
    st4<R, VEC>(y, c, a);
  }, [&](long long i) {
    R a = y[i];
    for (int qq = 0; qq < k; ++qq) a -= cf[qq] * X[qq * ld + i];
    y[i] = a * sc;
  });
}

__global__ void k_sqrt_store(const double* in, double* out) { *out = sqrt(fmax(*in, 0.0)); }

}  // namespace

// Packets need every pointer 16-byte aligned and, for a multivector, a leading
// dimension that keeps each column aligned.
template <typename R>
inline bool mv_aligned(const R* X, long long ld) {
  return al16(X) && ((ld * (long long)sizeof(R)) & 15) == 0;
}

template <typename Rd, typename Rs>
void vcast(long long n, const Rs* x, Rd* y, cudaStream_t s) {
  if (al16(x) && al16(y))
    k_cast<Rd, Rs, true><<<map_blocks(n), VT, 0, s>>>(n, x, y);
  else
    k_cast<Rd, Rs, false><<<map_blocks(n), VT, 0, s>>>(n, x, y);
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
  if (al16(x) && al16(y))
    k_axpy<R, true><<<map_blocks(n), VT, 0, s>>>(n, a, x, y);
  else
    k_axpy<R, false><<<map_blocks(n), VT, 0, s>>>(n, a, x, y);
}
template <typename R>
void vxpay(long long n, const R* x, R a, R* y, cudaStream_t s) {
  if (al16(x) && al16(y))
    k_xpay<R, true><<<map_blocks(n), VT, 0, s>>>(n, x, a, y);
  else
    k_xpay<R, false><<<map_blocks(n), VT, 0, s>>>(n, x, a, y);
}
template <typename R>
void vwaxpy(long long n, const R* x, R a, const R* y, R* w, cudaStream_t s) {
  if (al16(x) && al16(y) && al16(w))
    k_waxpy<R, true><<<map_blocks(n), VT, 0, s>>>(n, x, a, y, w);
  else
    k_waxpy<R, false><<<map_blocks(n), VT, 0, s>>>(n, x, a, y, w);
}
template <typename R>
void vdiv(long long n, const R* x, const R* d, R* y, cudaStream_t s) {
  if (al16(x) && al16(d) && al16(y))
    k_div<R, true><<<map_blocks(n), VT, 0, s>>>(n, x, d, y);
  else
    k_div<R, false><<<map_blocks(n), VT, 0, s>>>(n, x, d, y);
}
template <typename R>
void vscal(long long n, R a, R* y, cudaStream_t s) {
  if (al16(y))
    k_scal<R, true><<<map_blocks(n), VT, 0, s>>>(n, a, y);
  else
    k_scal<R, false><<<map_blocks(n), VT, 0, s>>>(n, a, y);
}
template <typename R>
void vscale_inv(long long n, const R* x, const double* nrm, R* y, cudaStream_t s) {
  if (al16(x) && al16(y))
    k_scale_inv<R, true><<<map_blocks(n), VT, 0, s>>>(n, x, nrm, y);
  else
    k_scale_inv<R, false><<<map_blocks(n), VT, 0, s>>>(n, x, nrm, y);
}

template <typename R>
static void mdot_partial(long long n, int k, const R* X, long long ld, const R* y, int self,
                         double* partial, int nb, cudaStream_t s) {
  if ((k == 0 || mv_aligned(X, ld)) && al16(y))
    k_mdot_partial<R, true><<<nb, RED_THREADS, 0, s>>>(n, k, X, ld, y, self, partial);
  else
    k_mdot_partial<R, false><<<nb, RED_THREADS, 0, s>>>(n, k, X, ld, y, self, partial);
}
template <typename R>
void vmdot(long long n, int k, const R* X, long long ld, const R* y, double* out, double* partial,
           cudaStream_t s) {
  const int nb = red_blocks(n);
  mdot_partial(n, k, X, ld, y, 0, partial, nb, s);
  k_mdot_final<<<k, RED_THREADS, 0, s>>>(nb, partial, out, 0);
}
template <typename R>
void vmdot_self(long long n, int k, const R* X, long long ld, const R* y, double* out,
                double* partial, cudaStream_t s) {
  const int nb = red_blocks(n);
  mdot_partial(n, k, X, ld, y, 1, partial, nb, s);
  k_mdot_final<<<k + 1, RED_THREADS, 0, s>>>(nb, partial, out, 0);
}
template <typename R>
void vnorm(long long n, const R* x, double* out, double* partial, cudaStream_t s) {
  const int nb = red_blocks(n);
  mdot_partial<R>(n, 0, nullptr, 0, x, 1, partial, nb, s);
  k_mdot_final<<<1, RED_THREADS, 0, s>>>(nb, partial, out, 1);
}
template <typename R>
void vinit_basis(long long n, const R* r, const R* D, R* v0, R* t, double* sig2_out,
                 double* partial, cudaStream_t s) {
  const int nb = red_blocks(n);
  if (al16(r) && al16(D) && al16(v0) && al16(t))
    k_init_basis<R, true><<<nb, RED_THREADS, 0, s>>>(n, r, D, v0, t, partial);
  else
    k_init_basis<R, false><<<nb, RED_THREADS, 0, s>>>(n, r, D, v0, t, partial);
  k_mdot_final<<<1, RED_THREADS, 0, s>>>(nb, partial, sig2_out, 0);
}
template <typename R>
void varnoldi_update(long long n, int k, const R* X, long long ld, const double* g,
                     const double* sig2, const R* D, R* w, R* t, double* sig2_out,
                     double* partial, cudaStream_t s) {
  const int nb = red_blocks(n);
  if (mv_aligned(X, ld) && al16(D) && al16(w) && al16(t))
    k_arnoldi_update<R, true><<<nb, RED_THREADS, 0, s>>>(n, k, X, ld, g, sig2, D, w, t, partial);
  else
    k_arnoldi_update<R, false><<<nb, RED_THREADS, 0, s>>>(n, k, X, ld, g, sig2, D, w, t, partial);
  k_mdot_final<<<1, RED_THREADS, 0, s>>>(nb, partial, sig2_out, 0);
}
template <typename R>
void vcombine(long long n, int k, const R* X, long long ld, const double* coef, const R* D, R* z,
              bool accumulate, cudaStream_t s) {
  if (mv_aligned(X, ld) && al16(D) && al16(z))
    k_combine<R, true><<<map_blocks(n), VT, 0, s>>>(n, k, X, ld, coef, D, z, accumulate ? 1 : 0);
  else
    k_combine<R, false><<<map_blocks(n), VT, 0, s>>>(n, k, X, ld, coef, D, z, accumulate ? 1 : 0);
}
template <typename R>
void vmaxpy(long long n, int k, const R* X, long long ld, const double* coef, double sign, R* y,
            cudaStream_t s) {
  if (mv_aligned(X, ld) && al16(y))
    k_maxpy<R, true><<<map_blocks(n), VT, 0, s>>>(n, k, X, ld, coef, sign, y);
  else
    k_maxpy<R, false><<<map_blocks(n), VT, 0, s>>>(n, k, X, ld, coef, sign, y);
}
template <typename R>
void vmaxpy_scale(long long n, int k, const R* X, long long ld, const double* h, const double* q,
                  double* nw_out, R* y, cudaStream_t s) {
  if (mv_aligned(X, ld) && al16(y))
    k_maxpy_scale<R, true><<<map_blocks(n), VT, 0, s>>>(n, k, X, ld, h, q, nw_out, y);
  else
    k_maxpy_scale<R, false><<<map_blocks(n), VT, 0, s>>>(n, k, X, ld, h, q, nw_out, y);
}
void vmaxpy_f32x(long long n, int k, const float* X, long long ld, const double* coef,
                 double sign, double* y, cudaStream_t s) {
  if (mv_aligned(X, ld) && al16(y))
    k_maxpy_f32x<true><<<map_blocks(n), VT, 0, s>>>(n, k, X, ld, coef, sign, y);
  else
    k_maxpy_f32x<false><<<map_blocks(n), VT, 0, s>>>(n, k, X, ld, coef, sign, y);
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
  template void vscale_inv<R>(long long, const R*, const double*, R*, cudaStream_t);           \
  template void vmdot<R>(long long, int, const R*, long long, const R*, double*, double*,      \
                         cudaStream_t);                                                        \
  template void vmdot_self<R>(long long, int, const R*, long long, const R*, double*, double*, \
                              cudaStream_t);                                                   \
  template void vnorm<R>(long long, const R*, double*, double*, cudaStream_t);                 \
  template void vinit_basis<R>(long long, const R*, const R*, R*, R*, double*, double*,        \
                               cudaStream_t);                                                  \
  template void varnoldi_update<R>(long long, int, const R*, long long, const double*,         \
                                   const double*, const R*, R*, R*, double*, double*,          \
                                   cudaStream_t);                                              \
  template void vcombine<R>(long long, int, const R*, long long, const double*, const R*, R*,  \
                            bool, cudaStream_t);                                               \
  template void vmaxpy<R>(long long, int, const R*, long long, const double*, double, R*,      \
                          cudaStream_t);                                                       \
  template void vmaxpy_scale<R>(long long, int, const R*, long long, const double*,            \
                                const double*, double*, R*, cudaStream_t);
NC_INST(double)
NC_INST(float)
#undef NC_INST

}  // namespace nc
