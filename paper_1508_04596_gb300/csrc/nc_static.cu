// Allocation-free Jacobian-vector product.
//
// nc_jvp needs a context from nc_setup, which allocates device memory (boundary
// flags, element scratch, multigrid workspace).  Some callers cannot allocate:
// an application whose memory pool has already reserved the device memory and
// forbids any other cudaMalloc, a plug-in that must not create allocations the
// host application does not track, or a latency-bound loop that cannot afford
// the implicit device synchronisation a cudaMalloc/cudaFree may cause.  For them,
// nc_jvp_static computes the same product with no allocation at all: its
// scratch (per-node boundary flags followed by the 40 element rows per
// element) lives in a file-scope device array of NC_STATIC_SCRATCH_BYTES that
// every GPU loading this library holds until the process exits.
//
// In host code the array's name is only a host-side stand-in for the device
// symbol, so its device address is looked up with cudaGetSymbolAddress, once per
// device, on the first call made with that device current.  Nothing in the
// scratch needs to start at zero: every flag and every element row is written
// before it is read, in stream order, within one call.  All calls share the one
// array, so two calls whose work overlaps on the GPU (different streams, or
// different host threads, without ordering between them) race on it.
#include <mutex>

#include "nc_internal.cuh"

using namespace nc;

namespace {

constexpr size_t kScratchBytes = NC_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Boundary flags of one node (bits 0..4: Dirichlet mask of u, v, w, p, T;
// bits 5..7: index of the Dirichlet temperature value), by the same face rules
// and precedence as nc_setup: velocity NOSLIP/SYMMETRY faces; temperature from
// the -x, +x, -y, +y faces, then the bottom patch, then -z, then +z.
struct FlagSpec {
  int vel_bc[6], T_bc[6];
  int patch_T;              // patch held at a temperature
  int pi0, pi1, pj0, pj1;   // patch node range on the bottom face
  long long pin;            // pinned pressure node or -1
};

__global__ void k_static_flags(LevelDev d, FlagSpec fs, uint8_t* flag) {
  const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= d.Nn) return;
  int i, j, k;
  node_ijk(d, n, i, j, k);
  const bool on[6] = {i == 0, i == d.nx, j == 0, j == d.ny, k == 0, k == d.nz};
  unsigned m = 0;
  for (int f = 0; f < 6; ++f) {
    if (!on[f]) continue;
    if (fs.vel_bc[f] == NC_VEL_NOSLIP) m |= 7u;
    else if (fs.vel_bc[f] == NC_VEL_SYMMETRY) m |= 1u << (f / 2);
  }
  int tv = 0;
  for (int f = 0; f < 4 && !tv; ++f)
    if (on[f] && fs.T_bc[f] == NC_T_DIRICHLET) tv = 1 + f;
  if (!tv && fs.patch_T && k == 0 && i >= fs.pi0 && i <= fs.pi1 && j >= fs.pj0 && j <= fs.pj1)
    tv = 5;
  if (!tv && on[4] && fs.T_bc[4] == NC_T_DIRICHLET) tv = 6;
  if (!tv && on[5] && fs.T_bc[5] == NC_T_DIRICHLET) tv = 7;
  if (tv) m |= 16u | (unsigned)(tv << 5);
  if (fs.pin == n) m |= 8u;
  flag[n] = (uint8_t)m;
}

// Patch node range on the bottom face, with the closed-interval test and the
// 1e-12 tolerance of nc_setup.
void patch_range(const nc_params& p, const nc_bcs& bc, int& pi0, int& pi1, int& pj0, int& pj1) {
  const double Lx = p.nx * p.h, Ly = p.ny * p.h;
  const double tol = 1e-12 * std::fmax(Lx, std::fmax(Ly, p.nz * p.h));
  const double x0 = bc.patch[0] * Lx, x1 = bc.patch[1] * Lx;
  const double y0 = bc.patch[2] * Ly, y1 = bc.patch[3] * Ly;
  pi0 = p.nx + 1; pi1 = -1; pj0 = p.ny + 1; pj1 = -1;
  for (int i = 0; i <= p.nx; ++i) {
    const double x = i * p.h;
    if (x >= x0 - tol && x <= x1 + tol) { if (i < pi0) pi0 = i; if (i > pi1) pi1 = i; }
  }
  for (int j = 0; j <= p.ny; ++j) {
    const double y = j * p.h;
    if (y >= y0 - tol && y <= y1 + tol) { if (j < pj0) pj0 = j; if (j > pj1) pj1 = j; }
  }
  if (pi0 > pi1 || pj0 > pj1) { pi0 = 0; pi1 = -1; pj0 = 0; pj1 = -1; }
}

}  // namespace

extern "C" nc_status nc_jvp_static(const nc_params* prm, const nc_bcs* bcs, const void* x,
                                   const void* gamma, const void* v, void* Jv, int prec,
                                   void* stream) {
  if (!prm || !bcs || !x || !gamma || !v || !Jv || (prec != NC_FP64 && prec != NC_FP32))
    return NC_ERR_ARG;
  // the checks of nc_setup: sizes bounded before any product of them is formed,
  // finite coefficients, face conditions, patch mode and pinned node in range
  std::string why;
  if (!valid_params(prm, why) || !valid_bcs(*prm, bcs, why)) return NC_ERR_ARG;
  LevelDev d;
  d.nx = prm->nx; d.ny = prm->ny; d.nz = prm->nz; d.h = prm->h;
  d.Nn = (long long)(d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  d.E = (long long)d.nx * d.ny * d.nz;
  // scratch: flags (Nn bytes, rounded up to 256), then the 40 element rows
  // (scratch_len(E) values)
  const size_t esz = prec == NC_FP64 ? sizeof(double) : sizeof(float);
  const size_t flag_bytes = ((size_t)d.Nn + 255) / 256 * 256;
  const double need = (double)flag_bytes + (double)scratch_len(d.E) * (double)esz;
  if (need > (double)kScratchBytes) return NC_ERR_SIZE;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return NC_ERR_CUDA;
  uint8_t* flag = (uint8_t*)base;
  void* Y = (unsigned char*)base + flag_bytes;

  FlagSpec fs;
  for (int f = 0; f < 6; ++f) { fs.vel_bc[f] = bcs->vel_bc[f]; fs.T_bc[f] = bcs->T_bc[f]; }
  fs.patch_T = bcs->patch_mode == NC_PATCH_DIRICHLET;
  patch_range(*prm, *bcs, fs.pi0, fs.pi1, fs.pj0, fs.pj1);
  fs.pin = bcs->p_pin;
  for (int q = 0; q < 8; ++q) d.tval[q] = 0.0;  // not used by J v
  d.patch_mode = bcs->patch_mode;
  d.pi0 = fs.pi0; d.pi1 = fs.pi1; d.pj0 = fs.pj0; d.pj1 = fs.pj1;
  d.q = bcs->patch_val;
  d.flag = flag;

  cudaStream_t s = (cudaStream_t)stream;
  k_static_flags<<<(unsigned)((d.Nn + 255) / 256), 256, 0, s>>>(d, fs, flag);
  if (prec == NC_FP64) {
    const ElemConst<double> c = make_const<double>(prm->h, prm->Gr, prm->Pr, prm->alpha_max,
                                                   prm->q_alpha, prm->q_f, prm->Ck, prm->g_dir);
    op_jvp<double>(d, c, (const double*)x, (const double*)gamma, nullptr, (const double*)v,
                   (double*)Jv, (double*)Y, s);
  } else {
    const ElemConst<float> c = make_const<float>(prm->h, prm->Gr, prm->Pr, prm->alpha_max,
                                                 prm->q_alpha, prm->q_f, prm->Ck, prm->g_dir);
    op_jvp<float>(d, c, (const float*)x, (const float*)gamma, nullptr, (const float*)v,
                  (float*)Jv, (float*)Y, s);
  }
  return cudaGetLastError() == cudaSuccess ? NC_OK : NC_ERR_CUDA;
}
