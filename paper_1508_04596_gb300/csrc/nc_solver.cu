// Solvers: Jacobi-preconditioned GMRES smoother, geometric multigrid V-cycle,
// flexible GMRES, damped Newton with the polynomial line search (Sec. 5.1) and
// the adjoint solve with FP64 iterative refinement (Sec. 3.2, Sec. 5.2).
//
// Precision: the outer FGMRES (Arnoldi with classical Gram-Schmidt applied
// twice, Hessenberg least squares on the host), the Newton residual, the
// refinement residual and every state update are FP64.  With mixed = 1 the
// Jacobian products inside FGMRES, the smoother and every multigrid level run
// in FP32; with mixed = 0 everything is FP64.
//
// The V-cycle and smoother run entirely on the device: their Hessenberg
// scalars stay in device memory and a one-thread kernel solves the small
// least-squares problem, so a preconditioner application never waits on the
// host.
#include <chrono>
#include <cmath>
#include <cstring>

#include "nc_internal.cuh"

namespace nc {
nc_status set_err(nc_ctx* ctx, nc_status st, const std::string& msg);
nc_status cuda_check(nc_ctx* ctx, cudaError_t e, const char* what);
}  // namespace nc

using namespace nc;

namespace {

constexpr int LDH = MAX_RESTART + 1;            // leading dimension of device Hessenbergs
constexpr int HD_Y = LDH * LDH;                   // y, then g, then the rotations
constexpr int HD_BETA = HD_Y + 4 * LDH;           // scalar slots
constexpr int HD_SIG2 = HD_BETA + 8;              // squared norms of the smoother basis
constexpr int HD_SIZE = HD_SIG2 + LDH;

template <typename R> LevelBuf<R>& buf(Level& L);
template <> LevelBuf<double>& buf<double>(Level& L) { return L.f64; }
template <> LevelBuf<float>& buf<float>(Level& L) { return L.f32; }
template <typename R> const ElemConst<R>& cst(const Level& L);
template <> const ElemConst<double>& cst<double>(const Level& L) { return L.c64; }
template <> const ElemConst<float>& cst<float>(const Level& L) { return L.c32; }

template <typename R>
nc_status alloc(nc_ctx* ctx, R** p, long long n) {
  if (*p) return NC_OK;
  return cuda_check(ctx, cudaMalloc((void**)p, sizeof(R) * (size_t)n), "cudaMalloc");
}

// Least squares of the smoother's Arnoldi process, on the device.  Column j of
// Hd holds the raw dots g_ij = <v_i, w_j> (i <= j) of the unnormalised basis
// v_i (squared norms sig2_i in Hd[HD_SIG2..]), built so that
//   A D^-1 v_j = sum_i g_ij / sig2_i v_i + sigma_j v_{j+1}.
// With q_i = v_i / sigma_i this is the usual Arnoldi relation with the
// Hessenberg entries H_ij = g_ij / (sigma_i sigma_j), H_{j+1,j} = sigma_{j+1},
// and beta = sigma_0.  Solve min || beta e1 - H y || by Givens rotations (in
// place), then store the coefficients of the correction on the raw basis,
// y_j / sigma_j -> Hd[HD_Y + j].  A vanishing norm or pivot (an exhausted
// Krylov space) contributes zero.  One warp stages the k columns and the norms
// in shared memory, then one thread solves there: the elimination is a chain of
// dependent operations, and in shared memory each costs tens of cycles instead
// of a round trip to L2.
constexpr int LS_THREADS = 32;
__global__ void __launch_bounds__(LS_THREADS) k_small_ls(double* Hd_g, int k) {
  __shared__ double Hd[HD_SIZE];
  for (int t = threadIdx.x; t < k * LDH; t += LS_THREADS) Hd[t] = Hd_g[t];
  for (int t = threadIdx.x; t <= k; t += LS_THREADS) Hd[HD_SIG2 + t] = Hd_g[HD_SIG2 + t];
  __syncwarp();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* g = Hd + HD_Y + LDH;  // right-hand side, k + 1 entries
  const double* sig2 = Hd + HD_SIG2;
  auto inv_sig = [&](int i) {
    const double s2 = sig2[i];
    return (s2 > 0.0 && s2 < 1e300) ? 1.0 / sqrt(s2) : 0.0;
  };
  const double beta = sqrt(fmax(sig2[0], 0.0));
  Hd[HD_BETA] = beta;
  for (int i = 0; i <= k; ++i) g[i] = 0.0;
  g[0] = (beta > 0.0 && beta < 1e300) ? beta : 0.0;
  for (int j = 0; j < k; ++j) {  // raw dots -> normalised Hessenberg
    double* hj = Hd + j * LDH;
    const double ij = inv_sig(j);
    for (int i = 0; i <= j; ++i) hj[i] *= inv_sig(i) * ij;
    hj[j + 1] = (ij > 0.0) ? sqrt(fmax(sig2[j + 1], 0.0)) : 0.0;
  }
  double rmax = 0.0;
  for (int j = 0; j < k; ++j) {
    double* hj = Hd + j * LDH;
    // apply the previous rotations (kept after g) to column j
    for (int q = 0; q < j; ++q) {
      const double c = Hd[HD_Y + 2 * LDH + 2 * q], s = Hd[HD_Y + 2 * LDH + 2 * q + 1];
      const double t1 = hj[q], t2 = hj[q + 1];
      hj[q] = c * t1 + s * t2;
      hj[q + 1] = -s * t1 + c * t2;
    }
    const double a = hj[j], b = hj[j + 1];
    const double r = hypot(a, b);
    const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? b / r : 0.0;
    Hd[HD_Y + 2 * LDH + 2 * j] = c;
    Hd[HD_Y + 2 * LDH + 2 * j + 1] = s;
    hj[j] = r;
    hj[j + 1] = 0.0;
    const double g1 = g[j], g2 = g[j + 1];
    g[j] = c * g1 + s * g2;
    g[j + 1] = -s * g1 + c * g2;
    rmax = fmax(rmax, fabs(r));
  }
  for (int j = k - 1; j >= 0; --j) {
    double acc = g[j];
    for (int q = j + 1; q < k; ++q) acc -= Hd[j + q * LDH] * Hd[HD_Y + q];
    const double d = Hd[j + j * LDH];
    Hd[HD_Y + j] = (fabs(d) > 1e-14 * rmax && isfinite(acc)) ? acc / d : 0.0;
  }
  for (int j = 0; j < k; ++j) Hd_g[HD_Y + j] = Hd[HD_Y + j] * inv_sig(j);
  Hd_g[HD_BETA] = Hd[HD_BETA];
}

// ------------------------------------------------------------------ level operators
template <typename R>
void level_apply(nc_ctx* ctx, int l, bool tr, const R* v, R* out, cudaStream_t s) {
  Level& L = ctx->lv[l];
  LevelBuf<R>& B = buf<R>(L);
  if (B.use_gst) {  // assembled or Galerkin operator
    op_stencil<R>(L.d, B.gst, tr, v, out, s);
    return;
  }
  if (B.lin) {  // FP64 levels: products from the linearisation cache
    if (tr)
      op_jtvp_cached<R>(L.d, cst<R>(L), B.x, B.gam, B.src, B.lin, v, out, (R*)ctx->Y, s);
    else
      op_jvp_cached<R>(L.d, cst<R>(L), B.x, B.gam, B.src, B.lin, v, out, (R*)ctx->Y, s);
    return;
  }
  if (tr)
    op_jtvp<R>(L.d, cst<R>(L), B.x, B.gam, B.src, v, out, (R*)ctx->Y, s);
  else
    op_jvp<R>(L.d, cst<R>(L), B.x, B.gam, B.src, v, out, (R*)ctx->Y, s);
}

// Right Jacobi-preconditioned GMRES(k) on level l:  z += D^-1 V y  approximately
// solving A z = b.  With zero_init the initial guess is 0.  The basis is kept
// unnormalised (each new vector is divided by the previous vector's norm, so
// magnitudes stay bounded); k_small_ls turns the raw dots and norms into the
// normalised Hessenberg.  Per Arnoldi step: the operator on t = D^-1 v_j, one
// multi-dot, and one pass that orthogonalises, rescales, forms the next t and
// the new norm.
template <typename R>
void smooth(nc_ctx* ctx, int l, bool tr, int k, bool zero_init, cudaStream_t s) {
  Level& L = ctx->lv[l];
  LevelBuf<R>& B = buf<R>(L);
  const long long n = 5 * L.d.Nn;
  const long long ld = mv_ld(n);
  R* V = B.V;
  double* Hd = B.Hd;
  if (zero_init) {
    vinit_basis(n, (const R*)B.b, (const R*)B.diag, V, B.t, Hd + HD_SIG2, ctx->partial, s);
  } else {
    level_apply<R>(ctx, l, tr, B.z, B.t, s);
    vwaxpy(n, (const R*)B.b, R(-1), (const R*)B.t, V, s);
    vinit_basis(n, (const R*)V, (const R*)B.diag, V, B.t, Hd + HD_SIG2, ctx->partial, s);
  }
  for (int j = 0; j < k; ++j) {
    R* w = V + (j + 1) * ld;
    level_apply<R>(ctx, l, tr, B.t, w, s);
    double* hcol = Hd + j * LDH;
    vmdot(n, j + 1, (const R*)V, ld, (const R*)w, hcol, ctx->partial, s);
    varnoldi_update(n, j + 1, (const R*)V, ld, hcol, Hd + HD_SIG2, (const R*)B.diag, w,
                    j + 1 < k ? B.t : (R*)nullptr, Hd + HD_SIG2 + j + 1, ctx->partial, s);
  }
  k_small_ls<<<1, LS_THREADS, 0, s>>>(Hd, k);
  // z (+)= D^-1 (V y)
  vcombine(n, k, (const R*)V, ld, Hd + HD_Y, (const R*)B.diag, B.z, !zero_init, s);
}

template <typename R>
void vcycle(nc_ctx* ctx, int l, int nlev, bool tr, const nc_solve_opts& o, cudaStream_t s) {
  Level& L = ctx->lv[l];
  LevelBuf<R>& B = buf<R>(L);
  if (l == nlev - 1) {
    if (B.inv)
      coarse_apply<R>(L, tr, B.inv, B.b, B.z, s);
    else
      smooth<R>(ctx, l, tr, o.coarse_its, true, s);
    return;
  }
  smooth<R>(ctx, l, tr, o.smooth_its, true, s);
  level_apply<R>(ctx, l, tr, B.z, B.t, s);
  vwaxpy(5 * L.d.Nn, (const R*)B.b, R(-1), (const R*)B.t, B.r, s);
  Level& C = ctx->lv[l + 1];
  op_restrict<R>(L.d, B.r, C.d, buf<R>(C).b, s);
  vcycle<R>(ctx, l + 1, nlev, tr, o, s);
  op_prolong_add<R>(C.d, buf<R>(C).z, L.d, B.z, s);
  smooth<R>(ctx, l, tr, o.smooth_its, false, s);
}

int n_levels(const nc_ctx* ctx, const nc_solve_opts& o) {
  int nl = (int)ctx->lv.size();
  if (o.mg_levels > 0 && o.mg_levels < nl) nl = o.mg_levels;
  return nl;
}

// Allocate the per-level workspace of precision R for nlev levels.
template <typename R>
nc_status alloc_levels(nc_ctx* ctx, int nlev, const nc_solve_opts& o) {
  nc_status st;
  for (int l = 0; l < nlev; ++l) {
    Level& L = ctx->lv[l];
    LevelBuf<R>& B = buf<R>(L);
    const long long n = 5 * L.d.Nn;
    const int ks = (l == nlev - 1) ? o.coarse_its : o.smooth_its;
    if (B.V && B.ks < ks) { cudaFree(B.V); B.V = nullptr; }
    if ((st = alloc(ctx, &B.V, (long long)(ks + 1) * mv_ld(n))) != NC_OK) return st;
    if (B.ks < ks) B.ks = ks;
    if ((st = alloc(ctx, &B.diag, n)) != NC_OK || (st = alloc(ctx, &B.b, n)) != NC_OK ||
        (st = alloc(ctx, &B.z, n)) != NC_OK || (st = alloc(ctx, &B.r, n)) != NC_OK ||
        (st = alloc(ctx, &B.t, n)) != NC_OK || (st = alloc(ctx, &B.Hd, (long long)HD_SIZE)) != NC_OK)
      return st;
    if (sizeof(R) == sizeof(double) &&
        (st = alloc(ctx, &B.lin, (long long)LIN_SLOTS * L.d.E)) != NC_OK)
      return st;
    if ((o.assembled || (o.galerkin && l >= 1)) &&
        (st = alloc(ctx, &B.gst, (long long)STENCIL_VALUES * L.d.Nn)) != NC_OK)
      return st;
    const bool level0_f64 = (l == 0) && sizeof(R) == sizeof(double);
    if (!level0_f64) {
      if ((st = alloc(ctx, &B.x, n)) != NC_OK || (st = alloc(ctx, &B.gam, L.d.E)) != NC_OK)
        return st;
    }
  }
  return NC_OK;
}

// Galerkin operator of level l >= 1 from level l - 1's operator, by probing
// (27 colours x 5 fields; see nc_galerkin.cu).
template <typename R>
void galerkin_build(nc_ctx* ctx, int l, cudaStream_t s) {
  Level& F = ctx->lv[l - 1];
  Level& L = ctx->lv[l];
  LevelBuf<R>& BF = buf<R>(F);
  LevelBuf<R>& BL = buf<R>(L);
  const long long nf = 5 * F.d.Nn;
  for (int c = 0; c < 27; ++c)
    for (int g = 0; g < 5; ++g) {
      galerkin_probe_init<R>(L.d, c, g, BL.t, s);
      vzero(nf, BF.t, s);
      op_prolong_add<R>(L.d, (const R*)BL.t, F.d, BF.t, s);
      level_apply<R>(ctx, l - 1, false, (const R*)BF.t, BF.r, s);
      op_restrict<R>(F.d, (const R*)BF.r, L.d, BL.r, s);
      galerkin_probe_scatter<R>(L.d, c, g, (const R*)BL.r, BL.gst, s);
    }
  stencil_dirichlet<R>(L.d, BL.gst, s);
}

// Linearisation data of every level in precision R at (x, gamma) (FP64 inputs):
// level 0 is x, gamma themselves (FP64) or their FP32 casts; coarser levels take
// the injected state and the mean design of the eight children and are
// rediscretised there, or (galerkin) hold P^T A P of the level above; with
// assembled, every rediscretised level's operator is assembled into a stencil;
// then diag(J).
template <typename R>
nc_status linearize(nc_ctx* ctx, int nlev, const double* x, const double* gam, cudaStream_t s,
                    const nc_solve_opts& o) {
  const bool galerkin = o.galerkin != 0, assembled = o.assembled != 0;
  for (int l = 0; l < nlev; ++l) {
    Level& L = ctx->lv[l];
    LevelBuf<R>& B = buf<R>(L);
    if (l == 0) {
      if (sizeof(R) == sizeof(double)) {
        L.f64.x = const_cast<double*>(x);
        L.f64.gam = const_cast<double*>(gam);
        L.f64.ext = true;
      } else {
        vcast(5 * L.d.Nn, x, (float*)B.x, s);
        vcast(L.d.E, gam, (float*)B.gam, s);
      }
    } else {
      Level& F = ctx->lv[l - 1];
      op_inject<R>(F.d, buf<R>(F).x, L.d, B.x, s);
      op_coarsen_elem<R>(F.d, buf<R>(F).gam, L.d, B.gam, s);
    }
    B.use_gst = assembled || (galerkin && l >= 1);
    if (galerkin && l >= 1) {
      galerkin_build<R>(ctx, l, s);
      op_stencil_diag<R>(L.d, B.gst, B.diag, s);
    } else if (assembled) {
      if (B.lin) op_linearize<R>(L.d, cst<R>(L), B.x, B.gam, B.src, B.lin, s);
      op_assemble<R>(L.d, cst<R>(L), B.x, B.gam, B.src, B.lin, B.gst, (R*)ctx->Y, s);
      op_stencil_diag<R>(L.d, B.gst, B.diag, s);
    } else {
      // diag(J^T) = diag(J)
      op_diag<R>(L.d, cst<R>(L), B.x, B.gam, B.src, B.diag, (R*)ctx->Y, s);
      if (B.lin) op_linearize<R>(L.d, cst<R>(L), B.x, B.gam, B.src, B.lin, s);
    }
    if (l == nlev - 1 && coarse_dense_dofs(L) <= COARSE_DENSE_MAX) {
      const nc_status st = B.use_gst ? coarse_setup_stencil<R>(ctx, L, B.gst, &B.inv, s)
                                     : coarse_setup<R>(ctx, L, B.x, B.gam, B.src, &B.inv, s);
      if (st != NC_OK) return st;
    } else if (B.inv) {
      cudaFree(B.inv);  // a previous solve used this level as the coarsest
      B.inv = nullptr;
    }
  }
  return NC_OK;
}

void release_ext(nc_ctx* ctx) {
  Level& L = ctx->lv[0];
  if (L.f64.ext) {
    L.f64.x = nullptr;
    L.f64.gam = nullptr;
    L.f64.ext = false;
  }
}

// ------------------------------------------------------------------ FGMRES (FP64)
struct LinSolve {
  bool tr = false;
  bool mixed = true;
  int nlev = 1;
};

// The V-cycle (level-0 b -> level-0 z) of one linear solve, captured once into a
// CUDA graph: a cycle is hundreds of small kernels on the coarse levels, and
// replaying the graph removes their per-launch host overhead.  If capture is
// not possible the cycle is launched kernel by kernel.
struct CycleGraph {
  cudaGraphExec_t exec = nullptr;
  ~CycleGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

void run_cycle(nc_ctx* ctx, const LinSolve& ls, const nc_solve_opts& o, cudaStream_t s) {
  if (ls.mixed)
    vcycle<float>(ctx, 0, ls.nlev, ls.tr, o, s);
  else
    vcycle<double>(ctx, 0, ls.nlev, ls.tr, o, s);
}

void capture_cycle(nc_ctx* ctx, const LinSolve& ls, const nc_solve_opts& o, CycleGraph& g) {
  if (!ctx->cap && cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking) != cudaSuccess) {
    ctx->cap = nullptr;
    cudaGetLastError();
    return;
  }
  if (cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  run_cycle(ctx, ls, o, ctx->cap);
  cudaGraph_t graph = nullptr;
  if (cudaStreamEndCapture(ctx->cap, &graph) != cudaSuccess || !graph) {
    cudaGetLastError();
    return;
  }
  if (cudaGraphInstantiate(&g.exec, graph, 0) != cudaSuccess) {
    cudaGetLastError();
    g.exec = nullptr;
  }
  cudaGraphDestroy(graph);
}

// z = M^-1 v (one V-cycle in the chosen precision); z is the FP64 column z64
// (FP64 solves) or the FP32 column z32 (mixed solves, whose cycle output is FP32)
void precond(nc_ctx* ctx, const LinSolve& ls, const nc_solve_opts& o, const CycleGraph& g,
             const double* v, double* z64, float* z32, cudaStream_t s) {
  Level& L = ctx->lv[0];
  const long long n = 5 * L.d.Nn;
  if (ls.mixed)
    vcast(n, v, L.f32.b, s);
  else
    vcopy(n, v, L.f64.b, s);
  if (g.exec)
    cudaGraphLaunch(g.exec, s);
  else
    run_cycle(ctx, ls, o, s);
  if (ls.mixed)
    vcopy(n, (const float*)L.f32.z, z32, s);
  else
    vcopy(n, (const double*)L.f64.z, z64, s);
}

// out = A z for an FP32 z (mixed solves: the FP32 product, its result in FP64)
void apply_A32(nc_ctx* ctx, const LinSolve& ls, const float* z, double* out, cudaStream_t s) {
  Level& L = ctx->lv[0];
  level_apply<float>(ctx, 0, ls.tr, z, L.f32.r, s);
  vcast(5 * L.d.Nn, (const float*)L.f32.r, out, s);
}

// out = A v with the linear solve's operator (FP32 product in mixed mode)
void apply_A(nc_ctx* ctx, const LinSolve& ls, const double* v, double* out, cudaStream_t s) {
  Level& L = ctx->lv[0];
  const long long n = 5 * L.d.Nn;
  if (ls.mixed) {
    vcast(n, v, L.f32.t, s);
    level_apply<float>(ctx, 0, ls.tr, L.f32.t, L.f32.r, s);
    vcast(n, (const float*)L.f32.r, out, s);
  } else {
    level_apply<double>(ctx, 0, ls.tr, v, out, s);
  }
}

nc_status read_scalar(nc_ctx* ctx, const double* d, double* h, int k, cudaStream_t s) {
  nc_status st = cuda_check(ctx, cudaMemcpyAsync(h, d, sizeof(double) * k, cudaMemcpyDeviceToHost, s),
                            "read scalar");
  if (st != NC_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(s), "stream sync");
}

nc_status norm2(nc_ctx* ctx, long long n, const double* v, double* out, cudaStream_t s) {
  vmdot(n, 1, v, 0, v, ctx->dscal, ctx->partial, s);
  double q;
  nc_status st = read_scalar(ctx, ctx->dscal, &q, 1, s);
  if (st != NC_OK) return st;
  *out = std::sqrt(std::fmax(q, 0.0));
  if (!std::isfinite(q)) return set_err(ctx, NC_ERR_NAN, "non-finite norm");
  return NC_OK;
}

// Classical Gram-Schmidt applied twice to w against the k orthonormal columns
// X_i = X + i*ld, with the normalisation folded into the second update: the
// second multi-dot also gives ||w1||^2, and ||w1 - X h2||^2 = ||w1||^2 - ||h2||^2
// (X orthonormal).  Device results: hc[0..k) = h1, hc[off..off+k) = h2,
// hc[off+k] = ||w1||^2, hc[2 off] = the final norm.  Four passes over the
// columns instead of six (two multi-dots, two updates, a norm and a scaling).
template <typename R>
void cgs2(long long n, int k, const R* X, long long ld, R* w, double* hc, int off,
          double* partial, cudaStream_t s) {
  double* h1 = hc;
  double* h2 = hc + off;
  vmdot(n, k, X, ld, (const R*)w, h1, partial, s);
  vmaxpy(n, k, X, ld, h1, 1.0, w, s);
  vmdot_self(n, k, X, ld, (const R*)w, h2, partial, s);
  vmaxpy_scale(n, k, X, ld, h2, h2 + k, hc + 2 * off, w, s);
}

// Solve A x = b to ||b - A x|| <= rtol ||b|| (x starts at 0).  its += iterations.
nc_status fgmres(nc_ctx* ctx, const LinSolve& ls, const nc_solve_opts& o, const double* b, double* x,
                 double rtol, int* its, cudaStream_t s) {
  Level& L = ctx->lv[0];
  const long long n = 5 * L.d.Nn;
  const int m = ctx->kry.m;
  const long long ld = mv_ld(n);
  double* V = ctx->kry.V;
  double* Z = ctx->kry.Z;    // FP64 solves
  float* Zf = ctx->kry.Zf;   // mixed solves
  double* hc = ctx->kry.hcol;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hh(2 * (m + 2) + 1);
  vzero(n, x, s);
  double beta0;
  nc_status st = norm2(ctx, n, b, &beta0, s);
  if (st != NC_OK) return st;
  if (beta0 == 0.0) return NC_OK;
  CycleGraph graph;
  capture_cycle(ctx, ls, o, graph);
  bool first = true;
  int total = 0;
  while (total < o.max_lin) {
    // r = b - A x  -> V0
    if (first) {
      vcopy(n, b, V, s);
    } else {
      apply_A(ctx, ls, x, ctx->kry.w, s);
      vwaxpy(n, b, -1.0, (const double*)ctx->kry.w, V, s);
    }
    double beta;
    if ((st = norm2(ctx, n, V, &beta, s)) != NC_OK) return st;
    if (beta <= rtol * beta0) break;
    vscal(n, 1.0 / beta, V, s);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    bool done = false;
    for (; j < m && total < o.max_lin; ++j) {
      double* vj = V + j * ld;
      double* w = V + (j + 1) * ld;
      if (ls.mixed) {
        float* zj = Zf + j * ld;
        precond(ctx, ls, o, graph, vj, nullptr, zj, s);
        apply_A32(ctx, ls, zj, w, s);
      } else {
        double* zj = Z + j * ld;
        precond(ctx, ls, o, graph, vj, zj, nullptr, s);
        apply_A(ctx, ls, zj, w, s);
      }
      cgs2(n, j + 1, (const double*)V, ld, w, hc, m + 2, ctx->partial, s);
      // one device-to-host read per iteration: both Gram-Schmidt columns and ||w||
      if ((st = read_scalar(ctx, hc, hh.data(), 2 * (m + 2) + 1, s)) != NC_OK) return st;
      const double nw = hh[2 * (m + 2)];
      if (!std::isfinite(nw) || !std::isfinite(hh[(m + 2) + j + 1]))
        return set_err(ctx, NC_ERR_NAN, "non-finite value in FGMRES");
      for (int i = 0; i <= j; ++i) H[i + (size_t)j * (m + 1)] = hh[i] + hh[(m + 2) + i];
      H[j + 1 + (size_t)j * (m + 1)] = nw;
      // apply previous rotations, then a new one
      for (int i = 0; i < j; ++i) {
        const double t1 = H[i + (size_t)j * (m + 1)], t2 = H[i + 1 + (size_t)j * (m + 1)];
        H[i + (size_t)j * (m + 1)] = cs[i] * t1 + sn[i] * t2;
        H[i + 1 + (size_t)j * (m + 1)] = -sn[i] * t1 + cs[i] * t2;
      }
      const double a = H[j + (size_t)j * (m + 1)], bb = H[j + 1 + (size_t)j * (m + 1)];
      const double r = std::hypot(a, bb);
      cs[j] = r > 0.0 ? a / r : 1.0;
      sn[j] = r > 0.0 ? bb / r : 0.0;
      H[j + (size_t)j * (m + 1)] = r;
      H[j + 1 + (size_t)j * (m + 1)] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      if (std::fabs(g[j + 1]) <= rtol * beta0 || nw == 0.0) {
        ++j;
        done = true;
        break;
      }
    }
    // y = H^-1 g, x += Z y
    std::vector<double> y(j);
    for (int i = j - 1; i >= 0; --i) {
      double acc = g[i];
      for (int q = i + 1; q < j; ++q) acc -= H[i + (size_t)q * (m + 1)] * y[q];
      const double d = H[i + (size_t)i * (m + 1)];
      y[i] = d != 0.0 ? acc / d : 0.0;
    }
    if (j > 0) {
      if ((st = cuda_check(ctx, cudaMemcpyAsync(ctx->kry.y, y.data(), sizeof(double) * j,
                                                cudaMemcpyHostToDevice, s), "upload y")) != NC_OK)
        return st;
      if (ls.mixed)
        vmaxpy_f32x(n, j, (const float*)Zf, ld, ctx->kry.y, -1.0, x, s);
      else
        vmaxpy(n, j, (const double*)Z, ld, ctx->kry.y, -1.0, x, s);
      if ((st = cuda_check(ctx, cudaStreamSynchronize(s), "fgmres sync")) != NC_OK) return st;
    }
    first = false;
    if (done) break;
  }
  *its += total;
  if (total >= o.max_lin) {
    // final check of the true residual
    apply_A(ctx, ls, x, ctx->kry.w, s);
    vwaxpy(n, b, -1.0, (const double*)ctx->kry.w, V, s);
    double rn;
    if ((st = norm2(ctx, n, V, &rn, s)) != NC_OK) return st;
    if (rn > rtol * beta0) return set_err(ctx, NC_ERR_MAXIT, "FGMRES reached max_lin");
  }
  return NC_OK;
}

nc_status prepare(nc_ctx* ctx, const nc_solve_opts& o, int nlev, bool mixed) {
  Level& L = ctx->lv[0];
  const long long n = 5 * L.d.Nn;
  nc_status st;
  if (o.restart < 1 || o.restart > MAX_RESTART || o.smooth_its < 1 ||
      o.smooth_its > MAX_RESTART || o.coarse_its < 1 || o.coarse_its > MAX_RESTART ||
      o.max_lin < 1 || o.max_newton < 0 || !(o.rtol_lin > 0.0) || !(o.rtol_newton >= 0.0) ||
      !(o.atol_newton >= 0.0) || !(o.rtol_adjoint >= 0.0) || o.adjoint_start < 0 ||
      o.adjoint_start > 1)
    return set_err(ctx, NC_ERR_ARG, "invalid solver options");
  if (ctx->kry.m < o.restart) {
    cudaFree(ctx->kry.V);
    cudaFree(ctx->kry.Z);
    cudaFree(ctx->kry.Zf);
    ctx->kry.V = ctx->kry.Z = nullptr;
    ctx->kry.Zf = nullptr;
    ctx->kry.m = 0;
  }
  if (!ctx->kry.V) {
    if ((st = alloc(ctx, &ctx->kry.V, (long long)(o.restart + 1) * mv_ld(n))) != NC_OK) return st;
    ctx->kry.m = o.restart;
  }
  // the preconditioned directions in the precision of the cycle that makes them
  // (allocated per mode at its first solve, sized by the current restart)
  if (mixed) {
    if ((st = alloc(ctx, &ctx->kry.Zf, (long long)ctx->kry.m * mv_ld(n))) != NC_OK) return st;
  } else {
    if ((st = alloc(ctx, &ctx->kry.Z, (long long)ctx->kry.m * mv_ld(n))) != NC_OK) return st;
  }
  if ((st = alloc(ctx, &ctx->kry.w, n)) != NC_OK ||
      (st = alloc(ctx, &ctx->kry.hcol, 2LL * (MAX_RESTART + 2) + 1)) != NC_OK ||
      (st = alloc(ctx, &ctx->kry.y, (long long)MAX_RESTART)) != NC_OK)
    return st;
  for (int i = 0; i < 6; ++i)
    if ((st = alloc(ctx, &ctx->tmp64[i], n)) != NC_OK) return st;
  if (mixed) {
    if ((st = alloc_levels<float>(ctx, nlev, o)) != NC_OK) return st;
  } else {
    if ((st = alloc_levels<double>(ctx, nlev, o)) != NC_OK) return st;
  }
  return NC_OK;
}

void set_Gr(nc_ctx* ctx, double Gr) {
  const nc_params& p = ctx->prm;
  for (auto& L : ctx->lv) {
    L.c64 = make_const<double>(L.d.h, Gr, p.Pr, p.alpha_max, p.q_alpha, p.q_f, p.Ck, p.g_dir);
    L.c32 = make_const<float>(L.d.h, Gr, p.Pr, p.alpha_max, p.q_alpha, p.q_f, p.Ck, p.g_dir);
  }
}

double line_search_length(double n0, double nh, double n1) {
  const double a = 2.0 * (n1 - 2.0 * nh + n0);
  const double b = n1 - n0 - a;
  if (a > 0.0) {
    const double lam = -b / (2.0 * a);
    if (lam > 0.0 && lam <= 1.0) return std::fmax(lam, 0.05);
  }
  return nh < n1 ? 0.5 : 1.0;
}

// Newton at the context's current Gr, from x (Dirichlet values already imposed),
// until ||R|| <= max(rtol ||R_0||, atol).  With stall_fails, three consecutive
// steps shorter than 0.1 that reduce ||R|| by less than 10 % count as a failure
// (NC_ERR_DIVERGED), which lets the caller switch to ramping.
nc_status newton(nc_ctx* ctx, const double* gam, double* x, const nc_solve_opts& o,
                 nc_solve_info* info, cudaStream_t s, double rtol, double atol,
                 bool stall_fails) {
  Level& L = ctx->lv[0];
  const long long n = 5 * L.d.Nn;
  const int nlev = n_levels(ctx, o);
  const bool mixed = o.mixed != 0;
  double* R = ctx->tmp64[0];
  double* d = ctx->tmp64[1];
  double* xt = ctx->tmp64[2];
  double* Rh = ctx->tmp64[3];
  double* R1 = ctx->tmp64[4];
  nc_status st;
  op_residual<double>(L.d, L.c64, x, gam, ctx->src64, R, ctx->Y, s);
  double nr;
  if ((st = norm2(ctx, n, R, &nr, s)) != NC_OK) return st;
  const double r0 = nr;
  if (info->newton_its == 0 && info->res0 == 0.0) info->res0 = r0;
  int it = 0;
  auto hist = [&](double v) {
    const int k = info->newton_its;
    if (k < 64) info->res_hist[k] = v;
  };
  if (info->newton_its == 0) hist(r0);
  const LinSolve ls{false, mixed, nlev};
  int stalls = 0;
  while (nr > std::fmax(rtol * r0, atol) && nr > 0.0) {
    if (it >= o.max_newton) {
      info->res_final = nr;
      return set_err(ctx, NC_ERR_MAXIT, "Newton reached max_newton");
    }
    st = mixed ? linearize<float>(ctx, nlev, x, gam, s, o)
               : linearize<double>(ctx, nlev, x, gam, s, o);
    if (st != NC_OK) return st;
    // J d = R, the Newton step is -d.  Inexact Newton: the linear solve goes to
    // rtol_lin (Sec. 5.2), or only as far as 0.01 of the Newton target where that
    // is looser (a last step that starts just above the target needs no 1e-5
    // reduction; with FP32 products a step reduces ||R|| by less than the linear
    // solve does, hence the margin).
    int lits = 0;
    const double eta = std::fmax(o.rtol_lin, std::fmin(0.01 * std::fmax(rtol * r0, atol) / nr, 0.5));
    st = fgmres(ctx, ls, o, R, d, eta, &lits, s);
    release_ext(ctx);
    info->lin_its_total += lits;
    if (st != NC_OK && st != NC_ERR_MAXIT) return st;
    vwaxpy(n, (const double*)x, -0.5, (const double*)d, xt, s);
    op_residual<double>(L.d, L.c64, xt, gam, ctx->src64, Rh, ctx->Y, s);
    double nh, n1;
    if ((st = norm2(ctx, n, Rh, &nh, s)) != NC_OK) return st;
    vwaxpy(n, (const double*)x, -1.0, (const double*)d, xt, s);
    op_residual<double>(L.d, L.c64, xt, gam, ctx->src64, R1, ctx->Y, s);
    if ((st = norm2(ctx, n, R1, &n1, s)) != NC_OK) return st;
    const double lam = line_search_length(nr, nh, n1);
    double nn;
    if (lam == 1.0) {
      vcopy(n, (const double*)xt, x, s);
      vcopy(n, (const double*)R1, R, s);
      nn = n1;
    } else if (lam == 0.5) {
      vaxpy(n, -0.5, (const double*)d, x, s);
      vcopy(n, (const double*)Rh, R, s);
      nn = nh;
    } else {
      vaxpy(n, -lam, (const double*)d, x, s);
      op_residual<double>(L.d, L.c64, x, gam, ctx->src64, R, ctx->Y, s);
      if ((st = norm2(ctx, n, R, &nn, s)) != NC_OK) return st;
    }
    ++it;
    ++info->newton_its;
    hist(nn);
    if (!(nn < nr) && !(std::fmin(nh, n1) < nr)) {
      nr = nn;
      info->res_final = nr;
      return set_err(ctx, NC_ERR_DIVERGED, "Newton: no decrease of the residual norm");
    }
    stalls = (lam <= 0.1 && nn > 0.9 * nr) ? stalls + 1 : 0;
    nr = nn;
    if (stall_fails && stalls >= 3) {
      info->res_final = nr;
      return set_err(ctx, NC_ERR_DIVERGED, "Newton: damped steps stagnate");
    }
  }
  info->res_final = nr;
  return NC_OK;
}

}  // namespace

extern "C" {

void nc_default_opts(nc_solve_opts* o) {
  if (!o) return;
  o->rtol_newton = 1e-8;
  o->rtol_lin = 1e-5;
  o->max_newton = 30;
  o->max_lin = 200;
  o->restart = 30;
  o->mg_levels = 0;
  o->smooth_its = 6;
  o->coarse_its = 30;
  o->mixed = 1;
  o->ramp_steps = 0;
  o->atol_newton = 0.0;
  o->galerkin = 0;
  o->assembled = 0;
  o->rtol_adjoint = 1e-10;
  o->adjoint_start = 0;
}

nc_status nc_newton_solve(nc_ctx* ctx, const double* gam, double* x, const nc_solve_opts* opts,
                          nc_solve_info* info_out, void* stream) {
  if (!ctx || !gam || !x) return set_err(ctx, NC_ERR_ARG, "nc_newton_solve: NULL argument");
  nc_solve_opts o;
  nc_default_opts(&o);
  if (opts) o = *opts;
  cudaStream_t s = (cudaStream_t)stream;
  nc_solve_info info;
  std::memset(&info, 0, sizeof(info));
  const auto t0 = std::chrono::steady_clock::now();
  const int nlev = n_levels(ctx, o);
  nc_status st = prepare(ctx, o, nlev, o.mixed != 0);
  if (st == NC_OK) {
    Level& L = ctx->lv[0];
    const long long n = 5 * L.d.Nn;
    op_impose<double>(L.d, x, s);
    // keep the start for a ramped retry
    if (o.ramp_steps > 0) vcopy(n, (const double*)x, ctx->tmp64[5], s);
    st = newton(ctx, gam, x, o, &info, s, o.rtol_newton, o.atol_newton, o.ramp_steps > 0);
    if (st != NC_OK && st != NC_ERR_ARG && st != NC_ERR_CUDA && st != NC_ERR_OOM &&
        o.ramp_steps > 0 && ctx->prm.Gr > 0.0) {
      // Sec. 5.1: recover from a failed start by ramping the load.  Here the
      // buoyancy is continued in log Gr from Gr / 10^steps: every stage starts
      // from the last converged state and is solved to 1e-4 of its own initial
      // residual (the paper's Newton tolerance); a stage that fails (or stalls)
      // is retried with half the step, a stage that converges lets the step grow
      // by half.  The last stage, at Gr itself, is solved to the requested
      // tolerance relative to the initial residual of the original problem.
      const double target = std::fmax(o.rtol_newton * info.res0, o.atol_newton);
      const double stage_rtol = std::fmax(o.rtol_newton, 1e-4);
      double* xlast = ctx->tmp64[5];  // the start, then the last converged stage
      const double lg_t = std::log10(ctx->prm.Gr);
      double lg = lg_t - o.ramp_steps;
      bool have = false;
      for (int tries = 0; tries < 4 && !have; ++tries, lg -= 1.0) {
        set_Gr(ctx, std::pow(10.0, lg));
        vcopy(n, (const double*)xlast, x, s);
        st = newton(ctx, gam, x, o, &info, s, stage_rtol, 0.0, true);
        have = st == NC_OK;
        if (!have && st != NC_ERR_MAXIT && st != NC_ERR_DIVERGED) break;
      }
      if (have) {
        lg += 1.0;  // undo the loop's last decrement
        vcopy(n, (const double*)x, xlast, s);
        double step = 1.0;
        int halvings = 0;
        while (lg < lg_t - 1e-12) {
          const double lg_try = std::fmin(lg + step, lg_t);
          const bool last = lg_try >= lg_t - 1e-12;
          set_Gr(ctx, last ? ctx->prm.Gr : std::pow(10.0, lg_try));
          vcopy(n, (const double*)xlast, x, s);
          st = last ? newton(ctx, gam, x, o, &info, s, 0.0, target, true)
                    : newton(ctx, gam, x, o, &info, s, stage_rtol, 0.0, true);
          if (st == NC_OK) {
            lg = lg_try;
            vcopy(n, (const double*)x, xlast, s);
            step *= 1.5;
          } else if ((st == NC_ERR_MAXIT || st == NC_ERR_DIVERGED) && ++halvings <= 8) {
            step *= 0.5;
          } else {
            break;
          }
        }
      }
      set_Gr(ctx, ctx->prm.Gr);
    }
  }
  release_ext(ctx);
  const nc_status st2 = cuda_check(ctx, cudaStreamSynchronize(s), "nc_newton_solve");
  if (st == NC_OK) st = st2;
  info.status = st;
  info.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info_out) *info_out = info;
  return st;
}

nc_status nc_arnoldi_orth(nc_ctx* ctx, long long n, int k, const void* V, long long ldv, void* w,
                          double* h_host, int prec, void* stream) {
  if (!ctx) return NC_ERR_ARG;
  if (!V || !w || !h_host || n < 1 || k < 1 || k > MAX_RESTART || ldv < n ||
      (prec != NC_FP64 && prec != NC_FP32))
    return set_err(ctx, NC_ERR_ARG, "nc_arnoldi_orth: invalid argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int off = MAX_RESTART + 2;
  double* hc = ctx->dscal;  // 2 * off + 1 slots
  if (prec == NC_FP64)
    cgs2(n, k, (const double*)V, ldv, (double*)w, hc, off, ctx->partial, s);
  else
    cgs2(n, k, (const float*)V, ldv, (float*)w, hc, off, ctx->partial, s);
  std::vector<double> hh(2 * off + 1);
  nc_status st = read_scalar(ctx, hc, hh.data(), 2 * off + 1, s);
  if (st != NC_OK) return st;
  for (int i = 0; i < k; ++i) h_host[i] = hh[i] + hh[off + i];
  h_host[k] = hh[2 * off];
  for (int i = 0; i <= k; ++i)
    if (!std::isfinite(h_host[i]) || !std::isfinite(hh[off + k]))
      return set_err(ctx, NC_ERR_NAN, "nc_arnoldi_orth: non-finite coefficient");
  return NC_OK;
}

nc_status nc_level_dims(nc_ctx* ctx, int level, int* dims) {
  if (!ctx) return NC_ERR_ARG;
  if (!dims || level < 0 || level >= (int)ctx->lv.size())
    return set_err(ctx, NC_ERR_ARG, "nc_level_dims: invalid level");
  dims[0] = ctx->lv[level].d.nx;
  dims[1] = ctx->lv[level].d.ny;
  dims[2] = ctx->lv[level].d.nz;
  return NC_OK;
}

nc_status nc_mg_apply(nc_ctx* ctx, int level, const double* x, const double* gam, const void* v,
                      void* out, int prec, int transpose, int galerkin, void* stream) {
  if (!ctx) return NC_ERR_ARG;
  if (!x || !gam || !v || !out || level < 0 || level >= (int)ctx->lv.size() ||
      (prec != NC_FP64 && prec != NC_FP32))
    return set_err(ctx, NC_ERR_ARG, "nc_mg_apply: invalid argument");
  nc_solve_opts o;
  nc_default_opts(&o);
  o.galerkin = galerkin != 0;
  const int nlev = level + 1;
  o.mg_levels = nlev;
  cudaStream_t s = (cudaStream_t)stream;
  const bool mixed = prec == NC_FP32;
  nc_status st = prepare(ctx, o, nlev, mixed);
  if (st != NC_OK) return st;
  st = mixed ? linearize<float>(ctx, nlev, x, gam, s, o)
             : linearize<double>(ctx, nlev, x, gam, s, o);
  if (st == NC_OK) {
    if (mixed)
      level_apply<float>(ctx, level, transpose != 0, (const float*)v, (float*)out, s);
    else
      level_apply<double>(ctx, level, transpose != 0, (const double*)v, (double*)out, s);
  }
  release_ext(ctx);
  const nc_status st2 = cuda_check(ctx, cudaStreamSynchronize(s), "nc_mg_apply");
  return st != NC_OK ? st : st2;
}

}  // extern "C"

namespace {
// FP64 linearisation store of the finest level for the mixed adjoint's
// refinement residuals (156 doubles per element), allocated on first use when
// the device keeps at least 8 GB free after it; false if it does not fit.
bool refine_store(nc_ctx* ctx, long long E) {
  if (ctx->ref_lin) return true;
  const size_t need = sizeof(double) * (size_t)LIN_SLOTS * (size_t)E;
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (fr < need + ((size_t)8 << 30)) return false;
  if (cudaMalloc((void**)&ctx->ref_lin, need) != cudaSuccess) {
    cudaGetLastError();
    ctx->ref_lin = nullptr;
    return false;
  }
  return true;
}
}  // namespace

extern "C" {

nc_status nc_adjoint_solve(nc_ctx* ctx, const double* x, const double* gam, const double* rhs,
                           double* lam, const nc_solve_opts* opts, nc_solve_info* info_out,
                           void* stream) {
  if (!ctx || !x || !gam || !rhs || !lam) return set_err(ctx, NC_ERR_ARG, "nc_adjoint_solve: NULL argument");
  nc_solve_opts o;
  nc_default_opts(&o);
  if (opts) o = *opts;
  cudaStream_t s = (cudaStream_t)stream;
  nc_solve_info info;
  std::memset(&info, 0, sizeof(info));
  const auto t0 = std::chrono::steady_clock::now();
  const int nlev = n_levels(ctx, o);
  const bool mixed = o.mixed != 0;
  nc_status st = prepare(ctx, o, nlev, mixed);
  if (st == NC_OK) {
    Level& L = ctx->lv[0];
    const long long n = 5 * L.d.Nn;
    double* r = ctx->tmp64[0];
    double* dl = ctx->tmp64[1];
    double* t = ctx->tmp64[2];
    double nb;
    st = norm2(ctx, n, rhs, &nb, s);
    info.res0 = nb;
    double nr = nb;
    // the state and the design do not change during the refinement: one
    // linearisation of every level serves all sweeps
    if (st == NC_OK)
      st = mixed ? linearize<float>(ctx, nlev, x, gam, s, o) : linearize<double>(ctx, nlev, x, gam, s, o);
    // FP64 refinement residuals r = rhs - J^T lam from an FP64 linearisation store
    // of the finest level: the FP64 solver's own, or in mixed mode one made here
    // when the device has room for it (else the state is re-interpolated)
    const double* store = nullptr;
    if (st == NC_OK) {
      if (!mixed) {
        store = L.f64.lin;
      } else if (refine_store(ctx, L.d.E)) {
        op_linearize<double>(L.d, L.c64, x, gam, ctx->src64, ctx->ref_lin, s);
        store = ctx->ref_lin;
      }
    }
    auto jt64 = [&](const double* w, double* out) {
      if (store)
        op_jtvp_cached<double>(L.d, L.c64, x, gam, ctx->src64, store, w, out, ctx->Y, s);
      else
        op_jtvp<double>(L.d, L.c64, x, gam, ctx->src64, w, out, ctx->Y, s);
    };
    if (st == NC_OK && o.adjoint_start) {  // warm start: the FP64 residual of the given lambda
      jt64(lam, t);
      vwaxpy(n, rhs, -1.0, (const double*)t, r, s);
      st = norm2(ctx, n, r, &nr, s);
    } else if (st == NC_OK) {
      vzero(n, lam, s);
      vcopy(n, rhs, r, s);
    }
    info.res_hist[0] = nr;
    const LinSolve ls{true, mixed, nlev};
    int k = 0;
    while (st == NC_OK && nr > o.rtol_adjoint * nb && nr > 0.0) {
      if (k >= o.max_newton) { st = set_err(ctx, NC_ERR_MAXIT, "adjoint refinement limit"); break; }
      int lits = 0;
      // inner relative tolerance: no tighter than needed for the outer target
      const double rt = std::fmax(o.rtol_lin, 0.5 * o.rtol_adjoint * nb / nr);
      st = fgmres(ctx, ls, o, r, dl, std::fmin(rt, 0.5), &lits, s);
      info.lin_its_total += lits;
      if (st != NC_OK && st != NC_ERR_MAXIT) break;
      vaxpy(n, 1.0, (const double*)dl, lam, s);
      // FP64 refinement residual r = rhs - J^T lam
      jt64(lam, t);
      vwaxpy(n, rhs, -1.0, (const double*)t, r, s);
      if ((st = norm2(ctx, n, r, &nr, s)) != NC_OK) break;
      ++k;
      if (k < 64) info.res_hist[k] = nr;
    }
    info.newton_its = k;
    info.res_final = nr;
  }
  release_ext(ctx);
  const nc_status st2 = cuda_check(ctx, cudaStreamSynchronize(s), "nc_adjoint_solve");
  if (st == NC_OK) st = st2;
  info.status = st;
  info.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info_out) *info_out = info;
  return st;
}

}  // extern "C"
