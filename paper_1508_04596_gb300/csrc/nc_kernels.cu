// Element operators, assembly by node-owner gather, and grid transfers.
//
// Assembly is colouring-free and deterministic: one thread per element writes
// its 40 element rows (f, a) to a scratch array (blocked by YB elements, see
// nc_internal.cuh); one thread per node then sums the rows of its (up to) eight
// elements in the fixed local order a = 0..7.  No atomics, so results are
// bitwise reproducible.
#include <type_traits>

#include "nc_element_f2.cuh"
#include "nc_internal.cuh"

namespace nc {

namespace {

constexpr int ELEM_THREADS = 128;
constexpr int NODE_THREADS = 256;

inline unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }


__device__ __forceinline__ long long node_id(const LevelDev& d, int i, int j, int k) {
  return i + (long long)(d.nx + 1) * (j + (long long)(d.ny + 1) * k);
}

template <typename R>
__device__ __forceinline__ void load_elem(const LevelDev& d, const R* __restrict__ x, long long e,
                                          R xe[5][8], bool mask) {
  int i, j, k;
  elem_ijk(d, e, i, j, k);
  const long long n0 = node_id(d, i, j, k);
  const long long sy = d.nx + 1, sz = (long long)(d.nx + 1) * (d.ny + 1);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const long long n = n0 + (a & 1) + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz;
    const uint8_t fl = mask ? d.flag[n] : uint8_t(0);
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      R v = x[f * d.Nn + n];
      xe[f][a] = (fl >> f) & 1 ? R(0) : v;
    }
  }
}

// node of local index a (bit 0: +x, bit 1: +y, bit 2: +z) of element e
__device__ __forceinline__ long long elem_node(const LevelDev& d, long long e, int a) {
  int i, j, k;
  elem_ijk(d, e, i, j, k);
  return node_id(d, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
}

// nodal velocities of the state (the only state data the cached products read)
template <typename R>
__device__ __forceinline__ void load_vel(const LevelDev& d, const R* __restrict__ x, long long e,
                                         R ue[3][8]) {
  const long long n0 = elem_node(d, e, 0);
  const long long sy = d.nx + 1, sz = (long long)(d.nx + 1) * (d.ny + 1);
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const long long n = n0 + (a & 1) + ((a >> 1) & 1) * sy + ((a >> 2) & 1) * sz;
#pragma unroll
    for (int f = 0; f < 3; ++f) ue[f][a] = x[f * d.Nn + n];
  }
}

// first row of element e in the blocked scratch; row r = 8 f + a is at + r YB
__device__ __forceinline__ long long yrow0(long long e) {
  static_assert(YB == 32, "yrow0 takes the block by a shift");
  return (e >> 5) * (40 * YB) + (e & (YB - 1));  // e >= 0
}

template <typename R>
__device__ __forceinline__ void store_elem(long long E, long long e, const R out[5][8], R* Y) {
  (void)E;
  R* y = Y + yrow0(e);
#pragma unroll
  for (int f = 0; f < 5; ++f)
#pragma unroll
    for (int a = 0; a < 8; ++a) y[(f * 8 + a) * YB] = out[f][a];
}

template <typename R>
__global__ void __launch_bounds__(ELEM_THREADS) k_elem_res(LevelDev d, ElemConst<R> c,
                                                           const R* __restrict__ x,
                                                           const R* __restrict__ gam,
                                                           const R* __restrict__ src, R* Y) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  R xe[5][8], out[5][8];
  load_elem(d, x, e, xe, false);
  elem_residual<R>(xe, gam[e], src ? src[e] : R(0), c, out);
  store_elem(d.E, e, out, Y);
}

// Two blocks per SM, up to 255 registers: both products then run without
// spilling.  J^T w, whose fluxes keep more values live, is 10 % faster in FP32
// than at three blocks (168 registers, spilled); J v, with fewer values live, is
// 1.5 % faster at 192x192x384 than at three blocks (where it spills 300 bytes a
// thread), 0.4 % at 128^3, and as fast as 64-thread blocks at five per SM.
// FP32 takes the packed-pair element routines (two lanes of FP32 arithmetic per
// instruction).  The nodal loads stay node by node with 64-bit indices: per-field
// base pointers with 32-bit row offsets cut the FP32 J v's instructions by 12 %
// but made it 10 % slower (more long-scoreboard stalls).
template <typename R, bool TRANSPOSE>
__global__ void __launch_bounds__(ELEM_THREADS, 2) k_elem_lin(LevelDev d, ElemConst<R> c,
                                                           const R* __restrict__ x,
                                                           const R* __restrict__ gam,
                                                           const R* __restrict__ src,
                                                           const R* __restrict__ v, R* Y) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  R xe[5][8], ve[5][8], out[5][8];
  load_elem(d, x, e, xe, false);
  load_elem(d, v, e, ve, true);  // Dirichlet columns removed
  const R g = gam[e], s = src ? src[e] : R(0);
  if constexpr (std::is_same<R, float>::value) {
    if (TRANSPOSE)
      elem_jtvp_f2(xe, ve, g, s, c, out);
    else
      elem_jvp_f2(xe, ve, g, s, c, out);
  } else {
    if (TRANSPOSE)
      elem_jtvp<R>(xe, ve, g, s, c, out);
    else
      elem_jvp<R>(xe, ve, g, s, c, out);
  }
  store_elem(d.E, e, out, Y);
}

template <typename R>
__global__ void __launch_bounds__(ELEM_THREADS) k_elem_linearize(LevelDev d, ElemConst<R> c,
                                                                 const R* __restrict__ x,
                                                                 const R* __restrict__ gam,
                                                                 const R* __restrict__ src,
                                                                 R* cache) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  R xe[5][8];
  load_elem(d, x, e, xe, false);
  elem_linearize<R>(xe, gam[e], src ? src[e] : R(0), c, cache + e, d.E);
}

// J v / J^T w from the linearisation cache: only the direction and the nodal
// velocities of the state are gathered.
template <typename R, bool TRANSPOSE>
__global__ void __launch_bounds__(ELEM_THREADS) k_elem_lin_cached(
    LevelDev d, ElemConst<R> c, const R* __restrict__ x, const R* __restrict__ gam,
    const R* __restrict__ src, const R* __restrict__ cache, const R* __restrict__ v, R* Y) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  R ue[3][8], ve[5][8], out[5][8];
  load_vel(d, x, e, ue);
  load_elem(d, v, e, ve, true);  // Dirichlet columns removed
  const R g = gam[e], s = src ? src[e] : R(0);
  if (TRANSPOSE)
    elem_jtvp_lin<R>(cache + e, d.E, ue, ve, g, s, c, out);
  else
    elem_jvp_lin<R>(cache + e, d.E, ue, ve, g, s, c, out);
  store_elem(d.E, e, out, Y);
}

// Column col = 5 b + g of every element Jacobian: the element product with the
// unit direction on unknown g of local node b, or zero where that unknown is
// Dirichlet (Dirichlet columns are removed).  Re-interpolates the state.
template <typename R>
__global__ void __launch_bounds__(ELEM_THREADS) k_elem_column(
    LevelDev d, ElemConst<R> c, const R* __restrict__ x, const R* __restrict__ gam,
    const R* __restrict__ src, int col, R* Y) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  const int b = col / 5, g = col % 5;
  R out[5][8];
  if ((d.flag[elem_node(d, e, b)] >> g) & 1) {
#pragma unroll
    for (int f = 0; f < 5; ++f)
#pragma unroll
      for (int a = 0; a < 8; ++a) out[f][a] = R(0);
    store_elem(d.E, e, out, Y);
    return;
  }
  R ve[5][8], xe[5][8];
#pragma unroll
  for (int f = 0; f < 5; ++f)
#pragma unroll
    for (int a = 0; a < 8; ++a) ve[f][a] = (f == g && a == b) ? R(1) : R(0);
  load_elem(d, x, e, xe, false);
  elem_jvp<R>(xe, ve, gam[e], src ? src[e] : R(0), c, out);
  store_elem(d.E, e, out, Y);
}

// The same column from the linearisation store with the unit direction written
// out (elem_column_lin): unknown G, local node b.
template <typename R, int G>
__global__ void __launch_bounds__(ELEM_THREADS) k_elem_column_lin(
    LevelDev d, ElemConst<R> c, const R* __restrict__ x, const R* __restrict__ gam,
    const R* __restrict__ src, const R* __restrict__ cache, int b, R* Y) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  R out[5][8];
  const long long nb = elem_node(d, e, b);
  if ((d.flag[nb] >> G) & 1) {
#pragma unroll
    for (int f = 0; f < 5; ++f)
#pragma unroll
      for (int a = 0; a < 8; ++a) out[f][a] = R(0);
  } else {
    const R ub = G < 3 ? x[G * d.Nn + nb] : R(0);
    elem_column_lin<R, G>(cache + e, d.E, ub, b, gam[e], src ? src[e] : R(0), c, out);
  }
  store_elem(d.E, e, out, Y);
}

// S += column col = 5 b + g of the element Jacobians, summed per node: row (n, f)
// takes entry (f, a) of each element e around n (n is e's local node a), at the
// stencil offset of e's local node b from n.  The eight elements around n give
// eight distinct offsets, so one launch writes no entry twice; the launches run
// in column order, so the sums are deterministic.  Dirichlet rows are skipped
// (they become identity rows afterwards).
template <typename R>
__global__ void __launch_bounds__(NODE_THREADS) k_assemble_column(LevelDev d, int col,
                                                                  const R* __restrict__ Y,
                                                                  R* __restrict__ S) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= d.Nn) return;
  int i, j, k;
  node_ijk(d, n, i, j, k);
  const int b = col / 5, g = col % 5;
  const uint8_t fl = d.flag[n];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int ie = i - (a & 1), je = j - ((a >> 1) & 1), ke = k - ((a >> 2) & 1);
    if (ie < 0 || je < 0 || ke < 0 || ie >= d.nx || je >= d.ny || ke >= d.nz) continue;
    const long long e = ie + (long long)d.nx * (je + (long long)d.ny * ke);
    const int o = ((b & 1) - (a & 1) + 1) + 3 * (((b >> 1) & 1) - ((a >> 1) & 1) + 1) +
                  9 * (((b >> 2) & 1) - ((a >> 2) & 1) + 1);
#pragma unroll
    for (int f = 0; f < 5; ++f)
      if (!((fl >> f) & 1)) S[((long long)(o * 5 + f) * 5 + g) * d.Nn + n] += Y[yrow0(e) + (f * 8 + a) * YB];
  }
}

template <typename R>
__global__ void __launch_bounds__(ELEM_THREADS) k_elem_diag(LevelDev d, ElemConst<R> c,
                                                            const R* __restrict__ x,
                                                            const R* __restrict__ gam,
                                                            const R* __restrict__ src, R* Y) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  R xe[5][8], out[5][8];
  load_elem(d, x, e, xe, false);
  elem_diag<R>(xe, gam[e], src ? src[e] : R(0), c, out);
  store_elem(d.E, e, out, Y);
}

__global__ void __launch_bounds__(ELEM_THREADS) k_elem_sens(LevelDev d, ElemConst<double> c,
                                                            const double* __restrict__ x,
                                                            const double* __restrict__ gam,
                                                            const double* __restrict__ src,
                                                            const double* __restrict__ lam,
                                                            double* out) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= d.E) return;
  double xe[5][8], le[5][8];
  load_elem(d, x, e, xe, false);
  load_elem(d, lam, e, le, true);  // Dirichlet rows excluded
  out[e] = elem_sens<double>(xe, le, gam[e], src ? src[e] : 0.0, c);
}

enum GatherMode { G_RES = 0, G_LIN = 1, G_DIAG = 2 };

__device__ __forceinline__ int patch_face_count(const LevelDev& d, int i, int j, int k) {
  if (d.patch_mode != NC_PATCH_FLUX || k != 0) return 0;
  int cnt = 0;
#pragma unroll
  for (int di = -1; di <= 0; ++di)
#pragma unroll
    for (int dj = -1; dj <= 0; ++dj) {
      const int ie = i + di, je = j + dj;
      cnt += (ie >= d.pi0 && ie <= d.pi1 - 1 && je >= d.pj0 && je <= d.pj1 - 1) ? 1 : 0;
    }
  return cnt;
}

template <typename R, int MODE>
__global__ void __launch_bounds__(NODE_THREADS) k_gather(LevelDev d, const R* __restrict__ Y,
                                                         const R* __restrict__ xv, R* out) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= d.Nn) return;
  int i, j, k;
  node_ijk(d, n, i, j, k);
  R acc[5] = {R(0), R(0), R(0), R(0), R(0)};
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int ie = i - (a & 1), je = j - ((a >> 1) & 1), ke = k - ((a >> 2) & 1);
    if (ie < 0 || je < 0 || ke < 0 || ie >= d.nx || je >= d.ny || ke >= d.nz) continue;
    const long long e = ie + (long long)d.nx * (je + (long long)d.ny * ke);
#pragma unroll
    for (int f = 0; f < 5; ++f) acc[f] += Y[yrow0(e) + (f * 8 + a) * YB];
  }
  const uint8_t fl = d.flag[n];
  if (MODE == G_RES) {
    const int pc = patch_face_count(d, i, j, k);
    if (pc) acc[4] -= R(d.q * d.h * d.h * 0.25 * pc);
  }
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    R v = acc[f];
    if ((fl >> f) & 1) {
      if (MODE == G_RES) {
        const R xd = (f == 4) ? R(d.tval[fl >> 5]) : R(0);
        v = xv[f * d.Nn + n] - xd;
      } else if (MODE == G_LIN) {
        v = xv[f * d.Nn + n];
      } else {
        v = R(1);
      }
    }
    out[f * d.Nn + n] = v;
  }
}

template <typename R, bool ZERO>
__global__ void k_impose(LevelDev d, R* x) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= d.Nn) return;
  const uint8_t fl = d.flag[n];
  if (!(fl & 31)) return;
#pragma unroll
  for (int f = 0; f < 5; ++f)
    if ((fl >> f) & 1) x[f * d.Nn + n] = (f == 4 && !ZERO) ? R(d.tval[fl >> 5]) : R(0);
}

__global__ void k_objective_grad(LevelDev d, double* g, double inv_area) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= (long long)(d.nx + 1) * (d.ny + 1)) return;  // bottom plane only
  const int i = (int)(n % (d.nx + 1));
  const int j = (int)(n / (d.nx + 1));
  int cnt = 0;
  for (int di = -1; di <= 0; ++di)
    for (int dj = -1; dj <= 0; ++dj) {
      const int ie = i + di, je = j + dj;
      cnt += (ie >= d.pi0 && ie <= d.pi1 - 1 && je >= d.pj0 && je <= d.pj1 - 1) ? 1 : 0;
    }
  g[4 * d.Nn + n] = cnt * d.h * d.h * 0.25 * inv_area;
}

// Gradient of the thermal compliance f = int s T dV: T rows get
// sum over the node's elements of s_e h^3 / 8 (int_e N_a dV = h^3/8), in a fixed
// element order.
__global__ void k_source_grad(LevelDev d, const double* __restrict__ src, double* g) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= d.Nn) return;
  int i, j, k;
  node_ijk(d, n, i, j, k);
  double acc = 0.0;
  for (int a = 0; a < 8; ++a) {
    const int ie = i - (a & 1), je = j - ((a >> 1) & 1), ke = k - ((a >> 2) & 1);
    if (ie < 0 || je < 0 || ke < 0 || ie >= d.nx || je >= d.ny || ke >= d.nz) continue;
    acc += src[ie + (long long)d.nx * (je + (long long)d.ny * ke)];
  }
  g[4 * d.Nn + n] = acc * d.h * d.h * d.h * 0.125;
}

// ---- transfers between a fine level and the next coarser one (factor 2)
// 1-D Q1 prolongation weight of coarse node I for fine node i: 1 if i == 2I,
// 1/2 if |i - 2I| == 1.
template <typename R>
__global__ void k_restrict(LevelDev f, const R* __restrict__ rf, LevelDev c, R* rc) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= c.Nn) return;
  int I, J, K;
  node_ijk(c, n, I, J, K);
  const uint8_t cfl = c.flag[n];
  R acc[5] = {R(0), R(0), R(0), R(0), R(0)};
  for (int dk = -1; dk <= 1; ++dk) {
    const int k = 2 * K + dk;
    if (k < 0 || k > f.nz) continue;
    const R wk = dk ? R(0.5) : R(1);
    for (int dj = -1; dj <= 1; ++dj) {
      const int j = 2 * J + dj;
      if (j < 0 || j > f.ny) continue;
      const R wj = dj ? R(0.5) : R(1);
      for (int di = -1; di <= 1; ++di) {
        const int i = 2 * I + di;
        if (i < 0 || i > f.nx) continue;
        const R w = wk * wj * (di ? R(0.5) : R(1));
        const long long m = node_id(f, i, j, k);
        const uint8_t ffl = f.flag[m];
#pragma unroll
        for (int q = 0; q < 5; ++q)
          if (!((ffl >> q) & 1)) acc[q] += w * rf[q * f.Nn + m];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) rc[q * c.Nn + n] = ((cfl >> q) & 1) ? R(0) : acc[q];
}

template <typename R>
__global__ void k_prolong_add(LevelDev c, const R* __restrict__ zc, LevelDev f, R* zf) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= f.Nn) return;
  int i, j, k;
  node_ijk(f, n, i, j, k);
  const uint8_t ffl = f.flag[n];
  const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1, k0 = k >> 1,
            k1 = (k + 1) >> 1;
  const R wi = (i & 1) ? R(0.5) : R(1), wj = (j & 1) ? R(0.5) : R(1), wk = (k & 1) ? R(0.5) : R(1);
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    if ((ffl >> q) & 1) continue;
    const R* z = zc + q * c.Nn;
    R acc;
    if (!(i & 1) && !(j & 1) && !(k & 1)) {
      acc = z[node_id(c, i0, j0, k0)];
    } else {
      acc = R(0);
      const int is[2] = {i0, i1}, js[2] = {j0, j1}, ks[2] = {k0, k1};
      const int ni = (i & 1) ? 2 : 1, nj = (j & 1) ? 2 : 1, nk = (k & 1) ? 2 : 1;
      for (int a = 0; a < nk; ++a)
        for (int b = 0; b < nj; ++b)
          for (int cc = 0; cc < ni; ++cc) acc += z[node_id(c, is[cc], js[b], ks[a])];
      acc *= wi * wj * wk;
    }
    zf[q * f.Nn + n] += acc;
  }
}

template <typename R>
__global__ void k_inject(LevelDev f, const R* __restrict__ xf, LevelDev c, R* xc) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= c.Nn) return;
  int I, J, K;
  node_ijk(c, n, I, J, K);
  const long long m = node_id(f, 2 * I, 2 * J, 2 * K);
#pragma unroll
  for (int q = 0; q < 5; ++q) xc[q * c.Nn + n] = xf[q * f.Nn + m];
}

template <typename R>
__global__ void k_coarsen_elem(LevelDev f, const R* __restrict__ gf, LevelDev c, R* gc) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= c.E) return;
  int I, J, K;
  elem_ijk(c, e, I, J, K);
  R acc = R(0);
  for (int a = 0; a < 8; ++a) {
    const int i = 2 * I + (a & 1), j = 2 * J + ((a >> 1) & 1), k = 2 * K + ((a >> 2) & 1);
    acc += gf[i + (long long)f.nx * (j + (long long)f.ny * k)];
  }
  gc[e] = acc * R(0.125);
}

}  // namespace

template <typename R>
void op_residual(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam, const R* src,
                 R* r, R* Y, cudaStream_t s) {
  k_elem_res<R><<<nblocks(d.E, ELEM_THREADS), ELEM_THREADS, 0, s>>>(d, c, x, gam, src, Y);
  k_gather<R, G_RES><<<nblocks(d.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(d, Y, x, r);
}

template <typename R>
void op_jvp(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam, const R* src,
            const R* v, R* out, R* Y, cudaStream_t s) {
  k_elem_lin<R, false><<<nblocks(d.E, ELEM_THREADS), ELEM_THREADS, 0, s>>>(d, c, x, gam, src, v, Y);
  k_gather<R, G_LIN><<<nblocks(d.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(d, Y, v, out);
}

template <typename R>
void op_jtvp(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam, const R* src,
             const R* w, R* out, R* Y, cudaStream_t s) {
  k_elem_lin<R, true><<<nblocks(d.E, ELEM_THREADS), ELEM_THREADS, 0, s>>>(d, c, x, gam, src, w, Y);
  k_gather<R, G_LIN><<<nblocks(d.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(d, Y, w, out);
}

template <typename R>
void op_linearize(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam, const R* src,
                  R* cache, cudaStream_t s) {
  k_elem_linearize<R><<<nblocks(d.E, ELEM_THREADS), ELEM_THREADS, 0, s>>>(d, c, x, gam, src, cache);
}

template <typename R>
void op_jvp_cached(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam,
                   const R* src, const R* cache, const R* v, R* out, R* Y, cudaStream_t s) {
  k_elem_lin_cached<R, false><<<nblocks(d.E, ELEM_THREADS), ELEM_THREADS, 0, s>>>(d, c, x, gam, src,
                                                                                 cache, v, Y);
  k_gather<R, G_LIN><<<nblocks(d.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(d, Y, v, out);
}

template <typename R>
void op_jtvp_cached(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam,
                    const R* src, const R* cache, const R* w, R* out, R* Y, cudaStream_t s) {
  k_elem_lin_cached<R, true><<<nblocks(d.E, ELEM_THREADS), ELEM_THREADS, 0, s>>>(d, c, x, gam, src,
                                                                                cache, w, Y);
  k_gather<R, G_LIN><<<nblocks(d.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(d, Y, w, out);
}

template <typename R>
void op_diag(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam, const R* src,
             R* out, R* Y, cudaStream_t s) {
  k_elem_diag<R><<<nblocks(d.E, ELEM_THREADS), ELEM_THREADS, 0, s>>>(d, c, x, gam, src, Y);
  k_gather<R, G_DIAG><<<nblocks(d.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(d, Y, x, out);
}

template <typename R>
void op_assemble(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam, const R* src,
                 const R* cache, R* S, R* Y, cudaStream_t s) {
  cudaMemsetAsync(S, 0, sizeof(R) * (size_t)STENCIL_VALUES * (size_t)d.Nn, s);
  const unsigned eb = nblocks(d.E, ELEM_THREADS);
  for (int col = 0; col < 40; ++col) {
    const int b = col / 5;
    if (cache) {
      switch (col % 5) {
        case 0: k_elem_column_lin<R, 0><<<eb, ELEM_THREADS, 0, s>>>(d, c, x, gam, src, cache, b, Y); break;
        case 1: k_elem_column_lin<R, 1><<<eb, ELEM_THREADS, 0, s>>>(d, c, x, gam, src, cache, b, Y); break;
        case 2: k_elem_column_lin<R, 2><<<eb, ELEM_THREADS, 0, s>>>(d, c, x, gam, src, cache, b, Y); break;
        case 3: k_elem_column_lin<R, 3><<<eb, ELEM_THREADS, 0, s>>>(d, c, x, gam, src, cache, b, Y); break;
        default: k_elem_column_lin<R, 4><<<eb, ELEM_THREADS, 0, s>>>(d, c, x, gam, src, cache, b, Y);
      }
    } else
      k_elem_column<R><<<eb, ELEM_THREADS, 0, s>>>(d, c, x, gam, src, col, Y);
    k_assemble_column<R><<<nblocks(d.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(d, col, Y, S);
  }
  stencil_dirichlet<R>(d, S, s);
}

void op_sens(const LevelDev& d, const ElemConst<double>& c, const double* x, const double* gam,
             const double* src, const double* lam, double* out, cudaStream_t s) {
  k_elem_sens<<<nblocks(d.E, ELEM_THREADS), ELEM_THREADS, 0, s>>>(d, c, x, gam, src, lam, out);
}

template <typename R>
void op_impose(const LevelDev& d, R* x, cudaStream_t s) {
  k_impose<R, false><<<nblocks(d.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(d, x);
}

template <typename R>
void op_mask(const LevelDev& d, R* x, cudaStream_t s) {
  k_impose<R, true><<<nblocks(d.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(d, x);
}

double patch_area(const LevelDev& d) {
  if (d.pi1 <= d.pi0 || d.pj1 <= d.pj0) return 0.0;
  return (double)(d.pi1 - d.pi0) * (double)(d.pj1 - d.pj0) * d.h * d.h;
}

void op_source_grad(const LevelDev& d, const double* src, double* g, cudaStream_t s) {
  cudaMemsetAsync(g, 0, sizeof(double) * 5 * d.Nn, s);
  k_source_grad<<<nblocks(d.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(d, src, g);
}

void op_objective_grad(const LevelDev& d, double* g, cudaStream_t s) {
  cudaMemsetAsync(g, 0, sizeof(double) * 5 * d.Nn, s);
  const double A = patch_area(d);
  if (A <= 0.0) return;
  const long long nb = (long long)(d.nx + 1) * (d.ny + 1);
  k_objective_grad<<<nblocks(nb, NODE_THREADS), NODE_THREADS, 0, s>>>(d, g, 1.0 / A);
}

template <typename R>
void op_restrict(const LevelDev& fine, const R* rf, const LevelDev& coarse, R* rc, cudaStream_t s) {
  k_restrict<R><<<nblocks(coarse.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(fine, rf, coarse, rc);
}
template <typename R>
void op_prolong_add(const LevelDev& coarse, const R* zc, const LevelDev& fine, R* zf,
                    cudaStream_t s) {
  k_prolong_add<R><<<nblocks(fine.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(coarse, zc, fine, zf);
}
template <typename R>
void op_inject(const LevelDev& fine, const R* xf, const LevelDev& coarse, R* xc, cudaStream_t s) {
  k_inject<R><<<nblocks(coarse.Nn, NODE_THREADS), NODE_THREADS, 0, s>>>(fine, xf, coarse, xc);
}
template <typename R>
void op_coarsen_elem(const LevelDev& fine, const R* gf, const LevelDev& coarse, R* gc,
                     cudaStream_t s) {
  k_coarsen_elem<R><<<nblocks(coarse.E, NODE_THREADS), NODE_THREADS, 0, s>>>(fine, gf, coarse, gc);
}

#define NC_INST(R)                                                                              \
  template void op_residual<R>(const LevelDev&, const ElemConst<R>&, const R*, const R*,        \
                               const R*, R*, R*, cudaStream_t);                                 \
  template void op_jvp<R>(const LevelDev&, const ElemConst<R>&, const R*, const R*, const R*,   \
                          const R*, R*, R*, cudaStream_t);                                      \
  template void op_jtvp<R>(const LevelDev&, const ElemConst<R>&, const R*, const R*, const R*,  \
                           const R*, R*, R*, cudaStream_t);                                     \
  template void op_diag<R>(const LevelDev&, const ElemConst<R>&, const R*, const R*, const R*,  \
                           R*, R*, cudaStream_t);                                               \
  template void op_linearize<R>(const LevelDev&, const ElemConst<R>&, const R*, const R*,       \
                                const R*, R*, cudaStream_t);                                    \
  template void op_jvp_cached<R>(const LevelDev&, const ElemConst<R>&, const R*, const R*,      \
                                 const R*, const R*, const R*, R*, R*, cudaStream_t);           \
  template void op_jtvp_cached<R>(const LevelDev&, const ElemConst<R>&, const R*, const R*,     \
                                  const R*, const R*, const R*, R*, R*, cudaStream_t);          \
  template void op_assemble<R>(const LevelDev&, const ElemConst<R>&, const R*, const R*,        \
                               const R*, const R*, R*, R*, cudaStream_t);                       \
  template void op_impose<R>(const LevelDev&, R*, cudaStream_t);                                \
  template void op_mask<R>(const LevelDev&, R*, cudaStream_t);                                  \
  template void op_restrict<R>(const LevelDev&, const R*, const LevelDev&, R*, cudaStream_t);   \
  template void op_prolong_add<R>(const LevelDev&, const R*, const LevelDev&, R*, cudaStream_t);\
  template void op_inject<R>(const LevelDev&, const R*, const LevelDev&, R*, cudaStream_t);     \
  template void op_coarsen_elem<R>(const LevelDev&, const R*, const LevelDev&, R*, cudaStream_t);
NC_INST(double)
NC_INST(float)
#undef NC_INST

}  // namespace nc
