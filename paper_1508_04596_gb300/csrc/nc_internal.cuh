// Internal structures and kernel launchers of libnc (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/nc.h"
#include "nc_element.cuh"

namespace nc {

constexpr int NF = 5;
constexpr int MAX_LEVELS = 16;
constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS_MAX = 608;  // 4 x 152 SMs
constexpr int MAX_RESTART = 64;
constexpr int MAX_DIM = 1 << 20;  // largest element count per direction

// Argument checks shared by nc_setup and nc_jvp_static (nc_api.cu): finite
// positive sizes and coefficients, every dimension <= MAX_DIM (checked before
// any product of them is formed), face conditions and the patch mode in range,
// the pinned node inside the grid.  why receives the reason of a rejection.
bool valid_params(const nc_params* p, std::string& why);
bool valid_bcs(const nc_params& p, const nc_bcs* b, std::string& why);

// Geometry and boundary data of one grid level, passed to kernels by value.
struct LevelDev {
  int nx, ny, nz;
  long long Nn, E;
  double h;
  const uint8_t* flag;  // per node: bits 0..4 Dirichlet field mask, bits 5..7 T value index
  double tval[8];       // Dirichlet temperature values by index
  int patch_mode;       // NC_PATCH_*
  int pi0, pi1, pj0, pj1;  // patch node index range on the bottom face (inclusive)
  double q;             // patch flux (NC_PATCH_FLUX)
};

#if defined(__CUDACC__)
// (i, j, k) of a linear index idx = i + n0 (j + n1 k) below total.  With total
// below 2^32 (every grid that fits a GPU's memory in practice) this takes 32-bit
// unsigned division, which costs a fraction of the 64-bit routine on the GPU;
// the test is the same for every thread of a launch, so it does not diverge.
__host__ __device__ __forceinline__ void split3(long long idx, long long total, int n0, int n1, int& i,
                                       int& j, int& k) {
  if (total <= 0xffffffffLL) {
    const unsigned u = (unsigned)idx, t = u / (unsigned)n0, kk = t / (unsigned)n1;
    i = (int)(u - t * (unsigned)n0);
    j = (int)(t - kk * (unsigned)n1);
    k = (int)kk;
  } else {
    const long long t = idx / n0;
    i = (int)(idx - t * n0);
    j = (int)(t % n1);
    k = (int)(t / n1);
  }
}
// element e = i + nx (j + ny k)
__host__ __device__ __forceinline__ void elem_ijk(const LevelDev& d, long long e, int& i, int& j, int& k) {
  split3(e, d.E, d.nx, d.ny, i, j, k);
}
// node n = i + (nx+1) (j + (ny+1) k)
__host__ __device__ __forceinline__ void node_ijk(const LevelDev& d, long long n, int& i, int& j, int& k) {
  split3(n, d.Nn, d.nx + 1, d.ny + 1, i, j, k);
}
#endif

template <typename R>
struct Vec {
  R* p = nullptr;
};

// Per level, per precision buffers used by the multigrid cycle.
template <typename R>
struct LevelBuf {
  R* x = nullptr;      // linearisation state (levels >= 1; level 0 points elsewhere)
  R* gam = nullptr;    // design
  R* src = nullptr;    // element source (may be null)
  R* diag = nullptr;   // diag(J)
  R* b = nullptr;      // cycle right-hand side
  R* z = nullptr;      // cycle solution
  R* r = nullptr;      // temporary residual
  R* t = nullptr;      // temporary
  R* V = nullptr;      // smoother Krylov basis, (ks+1) vectors
  R* H = nullptr;      // unused for R = float (scalars are kept in double, see Hd)
  double* Hd = nullptr;  // device scalars: Hessenberg (MAX_RESTART+1)^2, y, beta, norms
  int ks = 0;
  bool ext = false;    // x and gam point to caller/Newton arrays (level 0, FP64)
  R* inv = nullptr;    // dense inverse of the level operator (coarsest level only)
  R* lin = nullptr;    // linearisation cache (FP64 levels)
  R* gst = nullptr;    // Galerkin coarse operator, 27-point stencil of 5x5 blocks (levels >= 1)
  bool use_gst = false;  // the current linearisation uses gst on this level
};

struct Level {
  LevelDev d;
  uint8_t* flag = nullptr;
  ElemConst<double> c64;
  ElemConst<float> c32;
  LevelBuf<double> f64;
  LevelBuf<float> f32;
};

struct Krylov {
  int m = 0;
  double* V = nullptr;   // (m+1) x ndof
  double* Z = nullptr;   // m x ndof: preconditioned directions (FP64 solves)
  float* Zf = nullptr;   // m x ndof: the same in mixed solves, where the V-cycle that
                         // produces them runs in FP32, so FP32 storage is exact
  double* w = nullptr;
  double* hcol = nullptr;  // device, 2*(m+2)
  double* y = nullptr;     // device, m
};

}  // namespace nc

struct nc_ctx {
  nc_params prm;
  nc_bcs bcs;
  std::vector<nc::Level> lv;
  double* Y = nullptr;        // element output scratch, scratch_len(E(level 0)) doubles
  double* partial = nullptr;  // reduction partials, (MAX_RESTART+2) * RED_BLOCKS_MAX doubles
  double* dscal = nullptr;    // device scalars for reductions (MAX_RESTART+2)
  double* src64 = nullptr;    // element source (level 0), FP64
  nc::Krylov kry;
  double* tmp64[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // FP64 [5][Nn]
  float* tmp32[2] = {nullptr, nullptr};
  int ws_ks = 0;              // smoother workspace size allocated
  double* cjel = nullptr;     // coarsest-level element Jacobians (40 x 40 per element)
  long long cjel_elems = 0;
  cudaStream_t cap = nullptr; // stream used to capture the V-cycle graph
  double* filt[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // filter CG
  double* pub_lin = nullptr;  // linearisation of nc_linearize (level 0, FP64)
  double* asm_lin = nullptr;  // linearisation used by nc_assemble (level 0, FP64)
  double* ref_lin = nullptr;  // linearisation of the mixed adjoint's FP64 refinement (level 0)
  const double* pub_x = nullptr;
  const double* pub_gam = nullptr;
  std::string err;
};

namespace nc {

// Element-row scratch: the 40 rows (f, a) of the element kernels, in blocks of
// YB consecutive elements: row r = 8 f + a of element e sits at
// Y[(e / YB) * 40 YB + r YB + e % YB].  A warp's 32 elements write each row as
// one contiguous 128-byte (FP32) or 256-byte (FP64) segment, and the 40 rows of an
// element lie at fixed offsets from its first (offsets known at compile time, so
// no per-row address arithmetic).  Holds 40 * round_up(E, YB) values.
constexpr int YB = 32;
inline long long scratch_len(long long E) { return 40 * ((E + YB - 1) / YB * YB); }

// ---- element operators (nc_kernels.cu); Y is scratch of scratch_len(E) elements of R
template <typename R>
void op_residual(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam, const R* src,
                 R* r, R* Y, cudaStream_t s);
template <typename R>
void op_jvp(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam, const R* src,
            const R* v, R* out, R* Y, cudaStream_t s);
template <typename R>
void op_jtvp(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam, const R* src,
             const R* w, R* out, R* Y, cudaStream_t s);
// linearisation cache (LIN_SLOTS values per element, slot-major) and the
// products that read it
template <typename R>
void op_linearize(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam, const R* src,
                  R* cache, cudaStream_t s);
template <typename R>
void op_jvp_cached(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam,
                   const R* src, const R* cache, const R* v, R* out, R* Y, cudaStream_t s);
template <typename R>
void op_jtvp_cached(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam,
                    const R* src, const R* cache, const R* w, R* out, R* Y, cudaStream_t s);
template <typename R>
void op_diag(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam, const R* src,
             R* out, R* Y, cudaStream_t s);
void op_sens(const LevelDev& d, const ElemConst<double>& c, const double* x, const double* gam,
             const double* src, const double* lam, double* out, cudaStream_t s);
template <typename R>
void op_impose(const LevelDev& d, R* x, cudaStream_t s);
template <typename R>
void op_mask(const LevelDev& d, R* x, cudaStream_t s);  // zero Dirichlet entries
void op_objective_grad(const LevelDev& d, double* dphidx, cudaStream_t s);
void op_source_grad(const LevelDev& d, const double* src, double* dphidx, cudaStream_t s);
double patch_area(const LevelDev& d);

// ---- transfers
template <typename R>
void op_restrict(const LevelDev& fine, const R* rf, const LevelDev& coarse, R* rc, cudaStream_t s);
template <typename R>
void op_prolong_add(const LevelDev& coarse, const R* zc, const LevelDev& fine, R* zf,
                    cudaStream_t s);
template <typename R>
void op_inject(const LevelDev& fine, const R* xf, const LevelDev& coarse, R* xc, cudaStream_t s);
template <typename R>
void op_coarsen_elem(const LevelDev& fine, const R* gf, const LevelDev& coarse, R* gc,
                     cudaStream_t s);

// ---- vector kernels (deterministic fixed-partition reductions)
template <typename Rd, typename Rs>
void vcast(long long n, const Rs* x, Rd* y, cudaStream_t s);
template <typename R>
void vcopy(long long n, const R* x, R* y, cudaStream_t s);
template <typename R>
void vzero(long long n, R* x, cudaStream_t s);
template <typename R>
void vaxpy(long long n, R a, const R* x, R* y, cudaStream_t s);  // y += a x
template <typename R>
void vxpay(long long n, const R* x, R a, R* y, cudaStream_t s);  // y = x + a y
template <typename R>
void vwaxpy(long long n, const R* x, R a, const R* y, R* w, cudaStream_t s);  // w = x + a y
template <typename R>
void vdiv(long long n, const R* x, const R* d, R* y, cudaStream_t s);  // y = x / d
template <typename R>
void vscal(long long n, R a, R* y, cudaStream_t s);  // y = a y
// Multivectors X_i = X + i*ld are stored with ld = mv_ld(n), a multiple of 64
// elements, so that every column starts on a 256-byte boundary.
inline long long mv_ld(long long n) { return (n + 63) / 64 * 64; }
// out[i] = <X_i, y> for i < k; result in device memory (double)
template <typename R>
void vmdot(long long n, int k, const R* X, long long ld, const R* y, double* out, double* partial,
           cudaStream_t s);
// as vmdot, and out[k] = <y, y> from the same pass
template <typename R>
void vmdot_self(long long n, int k, const R* X, long long ld, const R* y, double* out,
                double* partial, cudaStream_t s);
// y -= sign * sum_i coef[i] X_i   (coef in device memory, double)
template <typename R>
void vmaxpy(long long n, int k, const R* X, long long ld, const double* coef, double sign, R* y,
            cudaStream_t s);
// y -= sign * sum_i coef[i] X_i for FP32 columns X and an FP64 y, accumulated in
// FP64 (each FP32 entry is exact in FP64, so this equals vmaxpy on the FP64 casts)
void vmaxpy_f32x(long long n, int k, const float* X, long long ld, const double* coef,
                 double sign, double* y, cudaStream_t s);
// y <- (y - sum_i h[i] X_i) / nw with nw = sqrt(*q - sum_i h[i]^2) (X orthonormal,
// *q = ||y||^2 before the update); nw -> *nw_out.  The second pass of classical
// Gram-Schmidt with its normalisation.
template <typename R>
void vmaxpy_scale(long long n, int k, const R* X, long long ld, const double* h, const double* q,
                  double* nw_out, R* y, cudaStream_t s);
// y = x * (1/ *nrm) with a breakdown guard (device scalar)
template <typename R>
void vscale_inv(long long n, const R* x, const double* nrm, R* y, cudaStream_t s);
void dev_sqrt_store(const double* in, double* out, cudaStream_t s);
// *out = ||x||_2
template <typename R>
void vnorm(long long n, const R* x, double* out, double* partial, cudaStream_t s);
// Smoother Arnoldi with an unnormalised basis.  vinit_basis: v0 = r (r may be v0
// itself), t = r / D, *sig2_out = ||r||^2.  varnoldi_update with the dots
// g[i] = <v_i, w> (i < k) and the squared norms sig2[i]:
// w <- (w - sum_i g[i]/sig2[i] v_i) / sqrt(sig2[k-1]), t = w / D (t may be null),
// *sig2_out = ||w||^2.
template <typename R>
void vinit_basis(long long n, const R* r, const R* D, R* v0, R* t, double* sig2_out,
                 double* partial, cudaStream_t s);
template <typename R>
void varnoldi_update(long long n, int k, const R* X, long long ld, const double* g,
                     const double* sig2, const R* D, R* w, R* t, double* sig2_out,
                     double* partial, cudaStream_t s);
// z = (sum_i coef[i] X_i) / D (D may be null: no division), or z += ... with accumulate
template <typename R>
void vcombine(long long n, int k, const R* X, long long ld, const double* coef, const R* D, R* z,
              bool accumulate, cudaStream_t s);

// ---- stencil operators (nc_galerkin.cu): assembled level operators and Galerkin
// coarse operators.  S holds 675 * Nn entries, S[((o*5 + f)*5 + g)*Nn + n] couples
// (n, f) to (n + offset o, g), o = (dx+1) + 3 (dy+1) + 9 (dz+1)
constexpr int STENCIL_VALUES = 675;
// S = J(x, gamma) of one level, from its element Jacobians (nc_kernels.cu): 40
// element products with unit directions (reading `cache` when not null), each
// summed into S per node; Dirichlet rows identity, Dirichlet columns zero.
template <typename R>
void op_assemble(const LevelDev& d, const ElemConst<R>& c, const R* x, const R* gam, const R* src,
                 const R* cache, R* S, R* Y, cudaStream_t s);
template <typename R>
void op_stencil(const LevelDev& d, const R* S, bool tr, const R* v, R* out, cudaStream_t s);
template <typename R>
void op_stencil_diag(const LevelDev& d, const R* S, R* out, cudaStream_t s);
template <typename R>
void galerkin_probe_init(const LevelDev& d, int c, int g, R* v, cudaStream_t s);
template <typename R>
void galerkin_probe_scatter(const LevelDev& d, int c, int g, const R* r, R* S, cudaStream_t s);
template <typename R>
void stencil_dirichlet(const LevelDev& d, R* S, cudaStream_t s);

// ---- coarsest-level direct solve (nc_coarse.cu)
constexpr int COARSE_DENSE_MAX = 1000;  // largest coarsest level solved by a dense inverse
int coarse_dense_dofs(const Level& L);
template <typename R>
nc_status coarse_setup(nc_ctx* ctx, Level& L, const R* x, const R* gam, const R* src, R** inv,
                       cudaStream_t s);
template <typename R>
void coarse_apply(const Level& L, bool tr, const R* inv, const R* b, R* z, cudaStream_t s);
// dense inverse of a level's Galerkin stencil operator
template <typename R>
nc_status coarse_setup_stencil(nc_ctx* ctx, Level& L, const R* S, R** inv, cudaStream_t s);

}  // namespace nc
