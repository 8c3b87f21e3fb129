// C-ABI entry points of libnc: context set-up (grid levels, boundary flags,
// workspace) and the operator calls.  Solvers live in nc_solver.cu.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "nc_internal.cuh"

using namespace nc;

namespace nc {
nc_status set_err(nc_ctx* ctx, nc_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}
nc_status cuda_check(nc_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return NC_OK;
  cudaGetLastError();
  return set_err(ctx, e == cudaErrorMemoryAllocation ? NC_ERR_OOM : NC_ERR_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}
}  // namespace nc

namespace nc {

bool valid_params(const nc_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return false; }
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) { why = "nx, ny, nz must be >= 1"; return false; }
  // bounded first, so that no product of the sizes below can overflow
  if (p->nx > MAX_DIM || p->ny > MAX_DIM || p->nz > MAX_DIM) {
    why = "nx, ny, nz must be <= 2^20";
    return false;
  }
  if (!(p->h > 0.0) || !std::isfinite(p->h)) { why = "h must be positive and finite"; return false; }
  const long long Nn = (long long)(p->nx + 1) * (p->ny + 1) * (p->nz + 1);
  if (Nn > (1LL << 40)) { why = "grid too large"; return false; }
  if (!(p->Pr > 0.0) || !std::isfinite(p->Pr)) { why = "Pr must be positive and finite"; return false; }
  if (!(p->Ck > 0.0) || !std::isfinite(p->Ck)) { why = "Ck must be positive and finite"; return false; }
  if (!(p->alpha_max >= 0.0) || !std::isfinite(p->alpha_max)) {
    why = "alpha_max must be >= 0 and finite";
    return false;
  }
  if (!std::isfinite(p->Gr)) { why = "Gr must be finite"; return false; }
  return true;
}

bool valid_bcs(const nc_params& p, const nc_bcs* b, std::string& why) {
  if (!b) { why = "bcs is NULL"; return false; }
  for (int f = 0; f < 6; ++f) {
    if (b->vel_bc[f] < 0 || b->vel_bc[f] > 2) { why = "vel_bc out of range"; return false; }
    if (b->T_bc[f] < 0 || b->T_bc[f] > 1) { why = "T_bc out of range"; return false; }
  }
  if (b->patch_mode < 0 || b->patch_mode > 2) { why = "patch_mode out of range"; return false; }
  if (b->p_pin >= (long long)(p.nx + 1) * (p.ny + 1) * (p.nz + 1)) {
    why = "p_pin outside the grid";
    return false;
  }
  return true;
}

}  // namespace nc

namespace {

// Boundary flags of one level: bits 0..4 Dirichlet per field, bits 5..7 index
// of the Dirichlet temperature value.  Precedence of temperature values:
// -x, +x, -y, +y faces, then the bottom patch, then -z, then +z.
void build_flags(int nx, int ny, int nz, double h, const nc_bcs& bc, long long pin,
                 std::vector<uint8_t>& fl, double tval[8], int& pi0, int& pi1, int& pj0,
                 int& pj1) {
  const long long sx = nx + 1, sy = ny + 1;
  const long long Nn = sx * sy * (nz + 1);
  fl.assign(Nn, 0);
  // T value table: 0 unused, 1..4 side faces, 5 patch, 6 bottom, 7 top
  for (int q = 0; q < 8; ++q) tval[q] = 0.0;
  for (int f = 0; f < 4; ++f) tval[1 + f] = bc.T_val[f];
  tval[5] = bc.patch_val;
  tval[6] = bc.T_val[4];
  tval[7] = bc.T_val[5];
  // patch node index range on the bottom face
  const double Lx = nx * h, Ly = ny * h;
  const double tol = 1e-12 * std::fmax(Lx, std::fmax(Ly, nz * h));
  const double x0 = bc.patch[0] * Lx, x1 = bc.patch[1] * Lx;
  const double y0 = bc.patch[2] * Ly, y1 = bc.patch[3] * Ly;
  pi0 = nx + 1; pi1 = -1; pj0 = ny + 1; pj1 = -1;
  for (int i = 0; i <= nx; ++i) {
    const double x = i * h;
    if (x >= x0 - tol && x <= x1 + tol) { if (i < pi0) pi0 = i; if (i > pi1) pi1 = i; }
  }
  for (int j = 0; j <= ny; ++j) {
    const double y = j * h;
    if (y >= y0 - tol && y <= y1 + tol) { if (j < pj0) pj0 = j; if (j > pj1) pj1 = j; }
  }
  const bool patch_T = bc.patch_mode == NC_PATCH_DIRICHLET;
  for (int k = 0; k <= nz; ++k)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        const long long n = i + sx * (j + sy * k);
        const bool on[6] = {i == 0, i == nx, j == 0, j == ny, k == 0, k == nz};
        uint8_t m = 0;
        for (int f = 0; f < 6; ++f) {
          if (!on[f]) continue;
          if (bc.vel_bc[f] == NC_VEL_NOSLIP) m |= 7;
          else if (bc.vel_bc[f] == NC_VEL_SYMMETRY) m |= (uint8_t)(1 << (f / 2));
        }
        int tv = 0;
        for (int f = 0; f < 4 && !tv; ++f)
          if (on[f] && bc.T_bc[f] == NC_T_DIRICHLET) tv = 1 + f;
        if (!tv && patch_T && k == 0 && i >= pi0 && i <= pi1 && j >= pj0 && j <= pj1) tv = 5;
        if (!tv && on[4] && bc.T_bc[4] == NC_T_DIRICHLET) tv = 6;
        if (!tv && on[5] && bc.T_bc[5] == NC_T_DIRICHLET) tv = 7;
        if (tv) m |= (uint8_t)(16 | (tv << 5));
        if (pin == n) m |= 8;
        fl[n] = m;
      }
  if (pi0 > pi1 || pj0 > pj1) { pi0 = 0; pi1 = -1; pj0 = 0; pj1 = -1; }
}

template <typename R>
nc_status dev_alloc(nc_ctx* ctx, R** p, long long n) {
  *p = nullptr;
  if (n <= 0) return NC_OK;
  return cuda_check(ctx, cudaMalloc((void**)p, sizeof(R) * (size_t)n), "cudaMalloc");
}

void free_level(Level& L) {
  cudaFree(L.flag);
  L.flag = nullptr;
  if (L.f64.ext) { L.f64.x = nullptr; L.f64.gam = nullptr; }
  for (auto* b : {&L.f64.x, &L.f64.gam, &L.f64.src, &L.f64.diag, &L.f64.b, &L.f64.z, &L.f64.r,
                  &L.f64.t, &L.f64.V, &L.f64.H}) { cudaFree(*b); *b = nullptr; }
  for (auto* b : {&L.f32.x, &L.f32.gam, &L.f32.src, &L.f32.diag, &L.f32.b, &L.f32.z, &L.f32.r,
                  &L.f32.t, &L.f32.V}) { cudaFree(*b); *b = nullptr; }
  cudaFree(L.f32.H);
  L.f32.H = nullptr;
  cudaFree(L.f64.Hd);
  cudaFree(L.f32.Hd);
  L.f64.Hd = L.f32.Hd = nullptr;
  cudaFree(L.f64.inv);
  cudaFree(L.f32.inv);
  L.f64.inv = nullptr;
  L.f32.inv = nullptr;
  cudaFree(L.f64.lin);
  cudaFree(L.f32.lin);
  L.f64.lin = nullptr;
  L.f32.lin = nullptr;
  cudaFree(L.f64.gst);
  cudaFree(L.f32.gst);
  L.f64.gst = nullptr;
  L.f32.gst = nullptr;
}

bool check_prec(int prec) { return prec == NC_FP64 || prec == NC_FP32; }

}  // namespace

extern "C" {

const char* nc_status_string(int st) {
  switch (st) {
    case NC_OK: return "ok";
    case NC_ERR_ARG: return "invalid argument";
    case NC_ERR_CUDA: return "CUDA error";
    case NC_ERR_OOM: return "out of device memory";
    case NC_ERR_NAN: return "non-finite value";
    case NC_ERR_MAXIT: return "iteration limit reached";
    case NC_ERR_DIVERGED: return "Newton line search found no decrease";
    case NC_ERR_SIZE: return "problem larger than the fixed scratch of nc_jvp_static";
    default: return "unknown status";
  }
}

nc_status nc_sizes(const nc_params* prm, long long* n_nodes, long long* n_elems, long long* n_dof) {
  std::string why;
  if (!valid_params(prm, why)) return NC_ERR_ARG;
  const long long Nn = (long long)(prm->nx + 1) * (prm->ny + 1) * (prm->nz + 1);
  if (n_nodes) *n_nodes = Nn;
  if (n_elems) *n_elems = (long long)prm->nx * prm->ny * prm->nz;
  if (n_dof) *n_dof = 5 * Nn;
  return NC_OK;
}

const char* nc_last_error(const nc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void nc_destroy(nc_ctx* ctx) {
  if (!ctx) return;
  for (auto& L : ctx->lv) free_level(L);
  cudaFree(ctx->Y);
  cudaFree(ctx->partial);
  cudaFree(ctx->dscal);
  cudaFree(ctx->src64);
  cudaFree(ctx->kry.V);
  cudaFree(ctx->kry.Z);
  cudaFree(ctx->kry.Zf);
  cudaFree(ctx->kry.w);
  cudaFree(ctx->kry.hcol);
  cudaFree(ctx->kry.y);
  for (auto& p : ctx->tmp64) cudaFree(p);
  for (auto& p : ctx->tmp32) cudaFree(p);
  cudaFree(ctx->cjel);
  for (auto& p : ctx->filt) cudaFree(p);
  cudaFree(ctx->pub_lin);
  cudaFree(ctx->ref_lin);
  cudaFree(ctx->asm_lin);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  delete ctx;
}

nc_status nc_setup(const nc_params* prm, const nc_bcs* bcs, nc_ctx** out) {
  if (!out) return NC_ERR_ARG;
  *out = nullptr;
  std::string why;
  if (!valid_params(prm, why) || !valid_bcs(*prm, bcs, why)) return NC_ERR_ARG;
  nc_ctx* ctx = new (std::nothrow) nc_ctx();
  if (!ctx) return NC_ERR_OOM;
  ctx->prm = *prm;
  ctx->bcs = *bcs;
  // level hierarchy: halve while all dimensions stay even and >= 2 elements remain
  int nx = prm->nx, ny = prm->ny, nz = prm->nz;
  double h = prm->h;
  nc_status st = NC_OK;
  // pressure pin: node (pi, pj, pk) of the finest grid; on coarser grids the
  // coarse node (pi >> l, pj >> l, pk >> l)
  long long pin_ijk[3] = {-1, -1, -1};
  if (bcs->p_pin >= 0) {
    pin_ijk[0] = bcs->p_pin % (nx + 1);
    pin_ijk[1] = (bcs->p_pin / (nx + 1)) % (ny + 1);
    pin_ijk[2] = bcs->p_pin / ((long long)(nx + 1) * (ny + 1));
  }
  int lvl = 0;
  while (true) {
    Level L;
    L.d.nx = nx; L.d.ny = ny; L.d.nz = nz; L.d.h = h;
    L.d.Nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
    L.d.E = (long long)nx * ny * nz;
    std::vector<uint8_t> fl;
    const long long pin = bcs->p_pin >= 0
        ? (pin_ijk[0] >> lvl) + (long long)(nx + 1) * ((pin_ijk[1] >> lvl) +
                                                        (long long)(ny + 1) * (pin_ijk[2] >> lvl))
        : -1;
    build_flags(nx, ny, nz, h, *bcs, pin, fl, L.d.tval, L.d.pi0, L.d.pi1, L.d.pj0, L.d.pj1);
    L.d.patch_mode = bcs->patch_mode;
    L.d.q = bcs->patch_val;
    if ((st = dev_alloc(ctx, &L.flag, L.d.Nn)) != NC_OK) { nc_destroy(ctx); return st; }
    if ((st = cuda_check(ctx, cudaMemcpy(L.flag, fl.data(), L.d.Nn, cudaMemcpyHostToDevice),
                         "cudaMemcpy flags")) != NC_OK) { free_level(L); nc_destroy(ctx); return st; }
    L.d.flag = L.flag;
    L.c64 = make_const<double>(h, prm->Gr, prm->Pr, prm->alpha_max, prm->q_alpha, prm->q_f,
                               prm->Ck, prm->g_dir);
    L.c32 = make_const<float>(h, prm->Gr, prm->Pr, prm->alpha_max, prm->q_alpha, prm->q_f,
                              prm->Ck, prm->g_dir);
    ctx->lv.push_back(L);
    if (ctx->lv.size() >= (size_t)MAX_LEVELS) break;
    if ((nx & 1) || (ny & 1) || (nz & 1) || nx < 4 || ny < 4 || nz < 4) break;
    nx /= 2; ny /= 2; nz /= 2; h *= 2.0;
    ++lvl;
  }
  const Level& L0 = ctx->lv[0];
  if ((st = dev_alloc(ctx, &ctx->Y, scratch_len(L0.d.E))) != NC_OK) { nc_destroy(ctx); return st; }
  if ((st = dev_alloc(ctx, &ctx->partial, (long long)(MAX_RESTART + 2) * RED_BLOCKS_MAX)) != NC_OK ||
      (st = dev_alloc(ctx, &ctx->dscal, (long long)(MAX_RESTART + 2) * 4)) != NC_OK) {
    nc_destroy(ctx);
    return st;
  }
  *out = ctx;
  return NC_OK;
}

nc_status nc_bc_flags(nc_ctx* ctx, unsigned char* flags_host) {
  if (!ctx || !flags_host) return set_err(ctx, NC_ERR_ARG, "nc_bc_flags: NULL argument");
  const Level& L = ctx->lv[0];
  return cuda_check(ctx, cudaMemcpy(flags_host, L.flag, L.d.Nn, cudaMemcpyDeviceToHost),
                    "nc_bc_flags");
}

nc_status nc_set_source(nc_ctx* ctx, const double* src, void* stream) {
  if (!ctx) return NC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long long E = ctx->lv[0].d.E;
  if (!src) {
    cudaFree(ctx->src64);
    ctx->src64 = nullptr;
    for (auto& L : ctx->lv) {
      cudaFree(L.f64.src); L.f64.src = nullptr;
      cudaFree(L.f32.src); L.f32.src = nullptr;
    }
    return NC_OK;
  }
  nc_status st;
  if (!ctx->src64 && (st = dev_alloc(ctx, &ctx->src64, E)) != NC_OK) return st;
  cudaMemcpyAsync(ctx->src64, src, sizeof(double) * E, cudaMemcpyDeviceToDevice, s);
  // per-level copies (coarse levels: mean of the eight children)
  for (size_t l = 0; l < ctx->lv.size(); ++l) {
    Level& L = ctx->lv[l];
    if (!L.f64.src && (st = dev_alloc(ctx, &L.f64.src, L.d.E)) != NC_OK) return st;
    if (!L.f32.src && (st = dev_alloc(ctx, &L.f32.src, L.d.E)) != NC_OK) return st;
    if (l == 0)
      vcopy(E, ctx->src64, L.f64.src, s);
    else
      op_coarsen_elem(ctx->lv[l - 1].d, (const double*)ctx->lv[l - 1].f64.src, L.d, L.f64.src, s);
    vcast(L.d.E, (const double*)L.f64.src, L.f32.src, s);
  }
  return cuda_check(ctx, cudaStreamSynchronize(s), "nc_set_source");
}

nc_status nc_impose_dirichlet(nc_ctx* ctx, void* x, int prec, void* stream) {
  if (!ctx || !x || !check_prec(prec)) return set_err(ctx, NC_ERR_ARG, "nc_impose_dirichlet: bad argument");
  const Level& L = ctx->lv[0];
  if (prec == NC_FP64) op_impose(L.d, (double*)x, (cudaStream_t)stream);
  else op_impose(L.d, (float*)x, (cudaStream_t)stream);
  return cuda_check(ctx, cudaGetLastError(), "nc_impose_dirichlet");
}

nc_status nc_residual(nc_ctx* ctx, const void* x, const void* gam, void* r, int prec, void* stream) {
  if (!ctx || !x || !gam || !r || !check_prec(prec))
    return set_err(ctx, NC_ERR_ARG, "nc_residual: bad argument");
  const Level& L = ctx->lv[0];
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == NC_FP64)
    op_residual(L.d, L.c64, (const double*)x, (const double*)gam, L.f64.src, (double*)r, ctx->Y, s);
  else
    op_residual(L.d, L.c32, (const float*)x, (const float*)gam, L.f32.src, (float*)r,
                (float*)ctx->Y, s);
  return cuda_check(ctx, cudaGetLastError(), "nc_residual");
}

nc_status nc_jvp(nc_ctx* ctx, const void* x, const void* gam, const void* v, void* Jv, int prec,
                 void* stream) {
  if (!ctx || !x || !gam || !v || !Jv || !check_prec(prec))
    return set_err(ctx, NC_ERR_ARG, "nc_jvp: bad argument");
  const Level& L = ctx->lv[0];
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == NC_FP64)
    op_jvp(L.d, L.c64, (const double*)x, (const double*)gam, L.f64.src, (const double*)v,
           (double*)Jv, ctx->Y, s);
  else
    op_jvp(L.d, L.c32, (const float*)x, (const float*)gam, L.f32.src, (const float*)v, (float*)Jv,
           (float*)ctx->Y, s);
  return cuda_check(ctx, cudaGetLastError(), "nc_jvp");
}

nc_status nc_jtvp(nc_ctx* ctx, const void* x, const void* gam, const void* w, void* JTw, int prec,
                  void* stream) {
  if (!ctx || !x || !gam || !w || !JTw || !check_prec(prec))
    return set_err(ctx, NC_ERR_ARG, "nc_jtvp: bad argument");
  const Level& L = ctx->lv[0];
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == NC_FP64)
    op_jtvp(L.d, L.c64, (const double*)x, (const double*)gam, L.f64.src, (const double*)w,
            (double*)JTw, ctx->Y, s);
  else
    op_jtvp(L.d, L.c32, (const float*)x, (const float*)gam, L.f32.src, (const float*)w,
            (float*)JTw, (float*)ctx->Y, s);
  return cuda_check(ctx, cudaGetLastError(), "nc_jtvp");
}

nc_status nc_diag(nc_ctx* ctx, const void* x, const void* gam, void* d, int prec, void* stream) {
  if (!ctx || !x || !gam || !d || !check_prec(prec))
    return set_err(ctx, NC_ERR_ARG, "nc_diag: bad argument");
  const Level& L = ctx->lv[0];
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == NC_FP64)
    op_diag(L.d, L.c64, (const double*)x, (const double*)gam, L.f64.src, (double*)d, ctx->Y, s);
  else
    op_diag(L.d, L.c32, (const float*)x, (const float*)gam, L.f32.src, (float*)d, (float*)ctx->Y, s);
  return cuda_check(ctx, cudaGetLastError(), "nc_diag");
}

nc_status nc_linearize(nc_ctx* ctx, const double* x, const double* gam, void* stream) {
  if (!ctx || !x || !gam) return set_err(ctx, NC_ERR_ARG, "nc_linearize: bad argument");
  const Level& L = ctx->lv[0];
  nc_status st;
  if (!ctx->pub_lin &&
      (st = dev_alloc(ctx, &ctx->pub_lin, (long long)LIN_SLOTS * L.d.E)) != NC_OK)
    return st;
  op_linearize<double>(L.d, L.c64, x, gam, L.f64.src, ctx->pub_lin, (cudaStream_t)stream);
  ctx->pub_x = x;
  ctx->pub_gam = gam;
  return cuda_check(ctx, cudaGetLastError(), "nc_linearize");
}

nc_status nc_jvp_lin(nc_ctx* ctx, const double* v, double* Jv, void* stream) {
  if (!ctx || !v || !Jv) return set_err(ctx, NC_ERR_ARG, "nc_jvp_lin: bad argument");
  if (!ctx->pub_x) return set_err(ctx, NC_ERR_ARG, "nc_jvp_lin: call nc_linearize first");
  const Level& L = ctx->lv[0];
  op_jvp_cached<double>(L.d, L.c64, ctx->pub_x, ctx->pub_gam, L.f64.src, ctx->pub_lin, v, Jv,
                        ctx->Y, (cudaStream_t)stream);
  return cuda_check(ctx, cudaGetLastError(), "nc_jvp_lin");
}

nc_status nc_jtvp_lin(nc_ctx* ctx, const double* w, double* JTw, void* stream) {
  if (!ctx || !w || !JTw) return set_err(ctx, NC_ERR_ARG, "nc_jtvp_lin: bad argument");
  if (!ctx->pub_x) return set_err(ctx, NC_ERR_ARG, "nc_jtvp_lin: call nc_linearize first");
  const Level& L = ctx->lv[0];
  op_jtvp_cached<double>(L.d, L.c64, ctx->pub_x, ctx->pub_gam, L.f64.src, ctx->pub_lin, w, JTw,
                         ctx->Y, (cudaStream_t)stream);
  return cuda_check(ctx, cudaGetLastError(), "nc_jtvp_lin");
}

nc_status nc_assemble(nc_ctx* ctx, const void* x, const void* gam, void* S, int prec,
                      void* stream) {
  if (!ctx || !x || !gam || !S || !check_prec(prec))
    return set_err(ctx, NC_ERR_ARG, "nc_assemble: bad argument");
  const Level& L = ctx->lv[0];
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == NC_FP64) {
    nc_status st;
    if (!ctx->asm_lin &&
        (st = dev_alloc(ctx, &ctx->asm_lin, (long long)LIN_SLOTS * L.d.E)) != NC_OK)
      return st;
    op_linearize<double>(L.d, L.c64, (const double*)x, (const double*)gam, L.f64.src,
                         ctx->asm_lin, s);
    op_assemble<double>(L.d, L.c64, (const double*)x, (const double*)gam, L.f64.src,
                        ctx->asm_lin, (double*)S, ctx->Y, s);
  } else {
    op_assemble<float>(L.d, L.c32, (const float*)x, (const float*)gam, L.f32.src, nullptr,
                       (float*)S, (float*)ctx->Y, s);
  }
  return cuda_check(ctx, cudaGetLastError(), "nc_assemble");
}

nc_status nc_stencil_apply(nc_ctx* ctx, const void* S, const void* v, void* out, int transpose,
                           int prec, void* stream) {
  if (!ctx || !S || !v || !out || !check_prec(prec))
    return set_err(ctx, NC_ERR_ARG, "nc_stencil_apply: bad argument");
  const Level& L = ctx->lv[0];
  cudaStream_t s = (cudaStream_t)stream;
  if (prec == NC_FP64)
    op_stencil<double>(L.d, (const double*)S, transpose != 0, (const double*)v, (double*)out, s);
  else
    op_stencil<float>(L.d, (const float*)S, transpose != 0, (const float*)v, (float*)out, s);
  return cuda_check(ctx, cudaGetLastError(), "nc_stencil_apply");
}

nc_status nc_coarsen_elem(nc_ctx* ctx, int level, const double* e_fine, double* e_coarse,
                          void* stream) {
  if (!ctx || !e_fine || !e_coarse || level < 1 || level >= (int)ctx->lv.size())
    return set_err(ctx, NC_ERR_ARG, "nc_coarsen_elem: bad argument");
  op_coarsen_elem<double>(ctx->lv[level - 1].d, e_fine, ctx->lv[level].d, e_coarse,
                          (cudaStream_t)stream);
  return cuda_check(ctx, cudaGetLastError(), "nc_coarsen_elem");
}

nc_status nc_prolong_state(nc_ctx* ctx, int level, const double* x_coarse, double* x_fine,
                           void* stream) {
  if (!ctx || !x_coarse || !x_fine || level < 1 || level >= (int)ctx->lv.size())
    return set_err(ctx, NC_ERR_ARG, "nc_prolong_state: bad argument");
  const LevelDev& f = ctx->lv[level - 1].d;
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(x_fine, 0, sizeof(double) * 5 * (size_t)f.Nn, s);
  op_prolong_add<double>(ctx->lv[level].d, x_coarse, f, x_fine, s);
  op_impose<double>(f, x_fine, s);
  return cuda_check(ctx, cudaGetLastError(), "nc_prolong_state");
}

nc_status nc_objective(nc_ctx* ctx, const double* x, double* phi_host, double* dphidx,
                       void* stream) {
  if (!ctx || !x || !phi_host) return set_err(ctx, NC_ERR_ARG, "nc_objective: bad argument");
  const Level& L = ctx->lv[0];
  cudaStream_t s = (cudaStream_t)stream;
  double* g = dphidx;
  nc_status st;
  if (!g) {
    if (!ctx->tmp64[3] && (st = dev_alloc(ctx, &ctx->tmp64[3], 5 * L.d.Nn)) != NC_OK) return st;
    g = ctx->tmp64[3];
  }
  if (L.d.patch_mode == NC_PATCH_NONE && ctx->src64)
    op_source_grad(L.d, ctx->src64, g, s);  // thermal compliance (Sec. 3.2)
  else
    op_objective_grad(L.d, g, s);  // mean patch temperature
  // Phi = <dPhi/dx, x> (both objectives are linear in T)
  vmdot(5 * L.d.Nn, 1, g, 0, x, ctx->dscal, ctx->partial, s);
  if ((st = cuda_check(ctx, cudaMemcpyAsync(phi_host, ctx->dscal, sizeof(double),
                                            cudaMemcpyDeviceToHost, s), "nc_objective")) != NC_OK)
    return st;
  return cuda_check(ctx, cudaStreamSynchronize(s), "nc_objective");
}

nc_status nc_sensitivity(nc_ctx* ctx, const double* x, const double* gam, const double* lam,
                         double* out, void* stream) {
  if (!ctx || !x || !gam || !lam || !out) return set_err(ctx, NC_ERR_ARG, "nc_sensitivity: bad argument");
  const Level& L = ctx->lv[0];
  op_sens(L.d, L.c64, x, gam, L.f64.src, lam, out, (cudaStream_t)stream);
  return cuda_check(ctx, cudaGetLastError(), "nc_sensitivity");
}

}  // extern "C"
