// ALU throughput probe: dependent FMA chains in FP32 or FP64.
//
// The element kernels of this library are bound by the FP32 / FP64 pipes, not by
// HBM, so their roofline is an arithmetic peak.  The peak is derived from the
// unit counts and the SM clock; this kernel measures what a plain stream of
// fused multiply-adds actually reaches on the device, as a check of that
// derivation.  Each thread runs NCHAIN independent chains acc = acc * a + b
// (independent so that the pipe, not the FMA latency, sets the rate), unrolled
// 16 times per loop trip so that loop overhead is about 2 % of the issued
// instructions, and writes the sum of its chains so that nothing is dead code.
#include "nc_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 16;

template <typename R>
__global__ void __launch_bounds__(kThreads) k_fma_chain(long long trips, R a, R b, R* out) {
  R acc[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) acc[i] = R(threadIdx.x + i) * R(1e-3);
  for (long long t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
#pragma unroll
      for (int i = 0; i < kChains; ++i) acc[i] = fma(acc[i], a, b);
  }
  R s = R(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += acc[i];
  out[blockIdx.x * (long long)kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" nc_status nc_fma_probe(int prec, int blocks, long long iters, void* out, void* stream) {
  if (!out || blocks < 1 || iters < kUnroll || iters % kUnroll != 0 ||
      (prec != NC_FP64 && prec != NC_FP32))
    return NC_ERR_ARG;
  const long long trips = iters / kUnroll;
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == NC_FP64)
    k_fma_chain<double><<<blocks, kThreads, 0, s>>>(trips, 0.999999, 1e-7, (double*)out);
  else
    k_fma_chain<float><<<blocks, kThreads, 0, s>>>(trips, 0.9999f, 1e-4f, (float*)out);
  return cudaGetLastError() == cudaSuccess ? NC_OK : NC_ERR_CUDA;
}
