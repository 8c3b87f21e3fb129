// Operators stored as a 27-point stencil of 5 x 5 blocks per node: the
// assembled Jacobian of a level (built from the element Jacobians in
// nc_kernels.cu) and the Galerkin-projection coarse operators of Sec. 5.2,
// A_c = P^T A_f P on every coarse level.
//
// P is the trilinear prolongation of the V-cycle (fine Dirichlet unknowns left
// at zero) and P^T its restriction (fine Dirichlet rows dropped, coarse
// Dirichlet rows zero), so A_c is exactly the product the cycle's transfers
// define.  Coarse node I couples only to nodes J with |I - J| <= 1 per axis
// (P reaches one fine node, A_f one more, P^T one more: |2I - 2J| <= 3).
// The stencil is built by probing: coarse nodes are coloured by their indices
// mod 3 per axis (27 colours, no two nodes of a colour within one stencil), and
// for every colour c and field g the probe vector (1 on field g of the colour-c
// nodes that are not Dirichlet in g) is prolonged, multiplied by the finer
// level's operator and restricted; entry (I, f) of the result is the coupling
// of (I, f) to (J, g) with J the colour-c node next to I.  Dirichlet columns are
// zero (the probes skip them) and Dirichlet rows become identity rows, the same
// blockdiag(A_II, I) convention as the matrix-free operators.
//
// Layout: S[((o * 5 + f) * 5 + g) * Nn + n], offset o = (dx+1) + 3 (dy+1) + 9 (dz+1).
#include "nc_internal.cuh"

namespace nc {

namespace {

constexpr int GT = 256;
// The product runs in a single partial wave on small grids (8 blocks of 256 per
// SM); blocks of 128 halve the imbalance between SMs.
constexpr int AT = 128;

__device__ __forceinline__ long long nid(const LevelDev& d, int i, int j, int k) {
  return i + (long long)(d.nx + 1) * (j + (long long)(d.ny + 1) * k);
}

__device__ __forceinline__ int colour(int i, int j, int k) { return i % 3 + 3 * (j % 3) + 9 * (k % 3); }

template <typename R>
__global__ void k_probe_init(LevelDev d, int c, int g, R* __restrict__ v) {
  const long long n = blockIdx.x * (long long)GT + threadIdx.x;
  if (n >= d.Nn) return;
  int i, j, k;
  node_ijk(d, n, i, j, k);
  const bool on = colour(i, j, k) == c && !((d.flag[n] >> g) & 1);
#pragma unroll
  for (int f = 0; f < 5; ++f) v[f * d.Nn + n] = (f == g && on) ? R(1) : R(0);
}

// per axis: the offset in {-1, 0, 1} to the neighbour whose index is cc mod 3
__device__ __forceinline__ int colour_offset(int cc, int ii) {
  const int o = ((cc - ii) % 3 + 3) % 3;
  return o == 2 ? -1 : o;
}

template <typename R>
__global__ void k_probe_scatter(LevelDev d, int c, int g, const R* __restrict__ r, R* __restrict__ S) {
  const long long n = blockIdx.x * (long long)GT + threadIdx.x;
  if (n >= d.Nn) return;
  int i, j, k;
  node_ijk(d, n, i, j, k);
  const int dx = colour_offset(c % 3, i % 3), dy = colour_offset((c / 3) % 3, j % 3),
            dz = colour_offset(c / 9, k % 3);
  if (i + dx < 0 || i + dx > d.nx || j + dy < 0 || j + dy > d.ny || k + dz < 0 || k + dz > d.nz)
    return;
  const int o = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
#pragma unroll
  for (int f = 0; f < 5; ++f) S[((long long)(o * 5 + f) * 5 + g) * d.Nn + n] = r[f * d.Nn + n];
}

template <typename R>
__global__ void k_stencil_dirichlet(LevelDev d, R* __restrict__ S) {
  const long long n = blockIdx.x * (long long)GT + threadIdx.x;
  if (n >= d.Nn) return;
  const uint8_t fl = d.flag[n];
#pragma unroll
  for (int f = 0; f < 5; ++f)
    if ((fl >> f) & 1) S[((long long)(13 * 5 + f) * 5 + f) * d.Nn + n] = R(1);
}

// out = S v (TR: out = S^T v): one thread per node, the 27 neighbours in a
// fixed order (deterministic).
template <typename R, bool TR>
__global__ void __launch_bounds__(AT) k_stencil_apply(LevelDev d, const R* __restrict__ S,
                                                      const R* __restrict__ v, R* __restrict__ out) {
  const long long n = blockIdx.x * (long long)AT + threadIdx.x;
  if (n >= d.Nn) return;
  int i, j, k;
  node_ijk(d, n, i, j, k);
  const long long Nn = d.Nn;
  R acc[5] = {R(0), R(0), R(0), R(0), R(0)};
#pragma unroll 1
  for (int o = 0; o < 27; ++o) {
    const int ii = i + o % 3 - 1, jj = j + (o / 3) % 3 - 1, kk = k + o / 9 - 1;
    if (ii < 0 || ii > d.nx || jj < 0 || jj > d.ny || kk < 0 || kk > d.nz) continue;
    const long long m = nid(d, ii, jj, kk);
    R vm[5];
#pragma unroll
    for (int g = 0; g < 5; ++g) vm[g] = v[g * Nn + m];
    if (!TR) {
      const R* s = S + (long long)(o * 25) * Nn + n;
#pragma unroll
      for (int f = 0; f < 5; ++f)
#pragma unroll
        for (int g = 0; g < 5; ++g) acc[f] += s[(f * 5 + g) * Nn] * vm[g];
    } else {
      // row m's entry pointing back to n: offset index 26 - o
      const R* s = S + (long long)((26 - o) * 25) * Nn + m;
#pragma unroll
      for (int f = 0; f < 5; ++f)
#pragma unroll
        for (int g = 0; g < 5; ++g) acc[f] += s[(g * 5 + f) * Nn] * vm[g];
    }
  }
#pragma unroll
  for (int f = 0; f < 5; ++f) out[f * Nn + n] = acc[f];
}

template <typename R>
__global__ void k_stencil_diag(LevelDev d, const R* __restrict__ S, R* __restrict__ out) {
  const long long n = blockIdx.x * (long long)GT + threadIdx.x;
  if (n >= d.Nn) return;
#pragma unroll
  for (int f = 0; f < 5; ++f) out[f * d.Nn + n] = S[((long long)(13 * 5 + f) * 5 + f) * d.Nn + n];
}

inline unsigned gblocks(long long n, int t = GT) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <typename R>
void op_stencil(const LevelDev& d, const R* S, bool tr, const R* v, R* out, cudaStream_t s) {
  if (tr)
    k_stencil_apply<R, true><<<gblocks(d.Nn, AT), AT, 0, s>>>(d, S, v, out);
  else
    k_stencil_apply<R, false><<<gblocks(d.Nn, AT), AT, 0, s>>>(d, S, v, out);
}

template <typename R>
void op_stencil_diag(const LevelDev& d, const R* S, R* out, cudaStream_t s) {
  k_stencil_diag<R><<<gblocks(d.Nn), GT, 0, s>>>(d, S, out);
}

template <typename R>
void galerkin_probe_init(const LevelDev& d, int c, int g, R* v, cudaStream_t s) {
  k_probe_init<R><<<gblocks(d.Nn), GT, 0, s>>>(d, c, g, v);
}

template <typename R>
void galerkin_probe_scatter(const LevelDev& d, int c, int g, const R* r, R* S, cudaStream_t s) {
  k_probe_scatter<R><<<gblocks(d.Nn), GT, 0, s>>>(d, c, g, r, S);
}

template <typename R>
void stencil_dirichlet(const LevelDev& d, R* S, cudaStream_t s) {
  k_stencil_dirichlet<R><<<gblocks(d.Nn), GT, 0, s>>>(d, S);
}

#define NC_INST(R)                                                                              \
  template void op_stencil<R>(const LevelDev&, const R*, bool, const R*, R*, cudaStream_t);      \
  template void op_stencil_diag<R>(const LevelDev&, const R*, R*, cudaStream_t);                \
  template void galerkin_probe_init<R>(const LevelDev&, int, int, R*, cudaStream_t);            \
  template void galerkin_probe_scatter<R>(const LevelDev&, int, int, const R*, R*, cudaStream_t);\
  template void stencil_dirichlet<R>(const LevelDev&, R*, cudaStream_t);
NC_INST(double)
NC_INST(float)
#undef NC_INST

}  // namespace nc
