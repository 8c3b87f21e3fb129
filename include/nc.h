/* nc.h -- C ABI of libnc: a single-GPU (GB300, sm_103a) solver for the stabilised
 * Q1-Q1 natural-convection equations used in "Large scale three-dimensional
 * topology optimisation of heat sinks cooled by natural convection"
 * (Alexandersen, Sigmund, Aage).
 *
 * Problem (Sec. 2, Eq. 1a-c), dimensionless:
 *   u.grad u - Pr div(grad u + grad u^T) + grad p = -alpha(gamma) u - Gr Pr^2 e^g T
 *   div u = 0
 *   u.grad T - div(K(gamma) grad T) = s
 * with the design interpolations of Sec. 3.1 (Eq. 7-8), discretised with
 * stabilised trilinear hexahedra on a structured grid (Sec. 4, App. B).
 *
 * Conventions shared by every call:
 *  - Grid: nx*ny*nz cubic elements of edge h; node n = i + (nx+1)(j + (ny+1)k),
 *    element e = i + nx(j + ny k); z is vertical.
 *  - State and vector arrays: structure of arrays [5][Nn] (u, v, w, p, T), Nn the
 *    node count; design and element arrays: [E].
 *  - Array arguments are DEVICE pointers owned by the caller, unless a name ends
 *    in _host.  Element type: double for NC_FP64, float for NC_FP32.
 *  - Calls enqueue work on `stream` (a cudaStream_t; NULL = legacy default stream)
 *    and return without synchronising, except where a call documents a host result.
 *  - Inputs are never modified, except arguments named *_inout.
 *  - Errors: every call returns an nc_status; nc_last_error(ctx) gives a message.
 *    The library never aborts and never prints.
 *  - Dirichlet rows: the residual row of a Dirichlet unknown is x - x_D; the
 *    Jacobian is blockdiag(J_II, I): Dirichlet columns are removed from the
 *    interior rows and Dirichlet rows are identity rows, so (J v)_D = v_D and
 *    (J^T w)_D = w_D.
 */
#ifndef NC_H
#define NC_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nc_ctx nc_ctx;

typedef enum {
  NC_OK = 0,
  NC_ERR_ARG = 1,      /* invalid argument (sizes, pointers, options) */
  NC_ERR_CUDA = 2,     /* a CUDA runtime call failed */
  NC_ERR_OOM = 3,      /* device allocation failed */
  NC_ERR_NAN = 4,      /* a non-finite value appeared in a norm */
  NC_ERR_MAXIT = 5,    /* iteration limit reached before the tolerance */
  NC_ERR_DIVERGED = 6, /* Newton line search found no decrease */
  NC_ERR_SIZE = 7      /* problem larger than the fixed scratch of nc_jvp_static */
} nc_status;

typedef enum { NC_FP64 = 0, NC_FP32 = 1 } nc_prec;

enum { NC_VEL_NOSLIP = 0, NC_VEL_FREE = 1, NC_VEL_SYMMETRY = 2 };
enum { NC_T_ADIABATIC = 0, NC_T_DIRICHLET = 1 };
enum { NC_PATCH_NONE = 0, NC_PATCH_DIRICHLET = 1, NC_PATCH_FLUX = 2 };

/* Physical and discretisation parameters (Sec. 2, Sec. 3.1, Sec. 6.1). */
typedef struct {
  int nx, ny, nz;     /* elements per direction, >= 1 */
  double h;           /* element edge length, > 0 */
  double Gr, Pr;      /* Grashof and Prandtl numbers (Sec. 2) */
  double alpha_max;   /* Brinkman impermeability of solid (Sec. 3.1, Eq. 8) */
  double q_alpha;     /* convexity of the alpha interpolation (Eq. 8) */
  double q_f;         /* convexity of the conductivity interpolation (Eq. 7) */
  double Ck;          /* k_f / k_s (Sec. 2); K(solid) = 1/Ck */
  double g_dir[3];    /* unit gravity direction e^g, e.g. (0,0,-1) */
} nc_params;

/* Boundary conditions of the cavity problems (Sec. 6.1: cold vertical and top
 * walls, insulated bottom, symmetry planes of the quarter domain, closed walls;
 * the benchmark cavities heat a patch of the bottom instead of a source block).
 * Per face, order (-x, +x, -y, +y, -z, +z).
 * Velocity: NC_VEL_NOSLIP (u = 0), NC_VEL_FREE (traction-free, natural),
 * NC_VEL_SYMMETRY (normal component 0).  Temperature: NC_T_ADIABATIC or
 * NC_T_DIRICHLET with value T_val[face].  A rectangular patch of the bottom face,
 * patch = {x0, x1, y0, y1} as fractions of the domain width (closed interval,
 * tolerance 1e-12 of the domain size), is either held at T = patch_val
 * (NC_PATCH_DIRICHLET) or heated by the inward flux q = patch_val
 * (NC_PATCH_FLUX, applied on the bottom faces whose four nodes lie in the
 * patch).  Dirichlet temperature precedence on shared nodes: -x, +x, -y, +y
 * faces, then the patch, then -z, then +z.  p_pin >= 0 pins the pressure of that
 * node to 0 (closed cavities); -1 for none. */
typedef struct {
  int vel_bc[6];
  int T_bc[6];
  double T_val[6];
  double patch[4];
  int patch_mode;
  double patch_val;
  long long p_pin;
} nc_bcs;

/* Sizes of the discrete problem (Sec. 4: trilinear hexahedra on a structured
 * grid, 5 unknowns per node; Sec. 6.2-6.4 quote the resulting unknown counts,
 * e.g. 5,281,605 for 80 x 160 x 80 elements): n_nodes = (nx+1)(ny+1)(nz+1),
 * n_elems = nx ny nz, n_dof = 5 n_nodes, computed without allocating anything.
 * Any output pointer may be NULL.  Returns NC_ERR_ARG for invalid sizes. */
nc_status nc_sizes(const nc_params* prm, long long* n_nodes, long long* n_elems,
                   long long* n_dof);

/* Create a context on the current CUDA device for the discretised problem of
 * Sec. 2 and Sec. 4 with the boundary conditions of Sec. 6.1 (bcs) and the
 * material interpolation of Sec. 3.1 (prm): boundary-condition flags, the
 * geometric multigrid hierarchy of Sec. 5.2 (halving while every dimension stays
 * even and at least 2 elements remain) and all operator workspace are allocated
 * here.  prm and bcs are copied; the caller keeps ownership of both.
 * NC_ERR_ARG for invalid parameters (non-positive sizes, h, Pr or Ck, a face
 * condition or patch mode out of range, a pinned node outside the grid),
 * NC_ERR_OOM if an allocation fails.
 * Krylov workspace is allocated at the first solve (sized by its restart).
 * On failure *out is NULL and the status says why. */
nc_status nc_setup(const nc_params* prm, const nc_bcs* bcs, nc_ctx** out);

/* Release every device allocation of the context.  NULL is accepted. */
void nc_destroy(nc_ctx* ctx);

/* Message of the last failed call on ctx (empty string if none; never NULL). */
const char* nc_last_error(const nc_ctx* ctx);

/* Static text for a status code. */
const char* nc_status_string(int status);

/* Per-node boundary flags computed by nc_setup, copied to host memory:
 * bit f (0..4) set if unknown f of the node is Dirichlet.  flags_host has Nn
 * bytes.  Synchronous. */
nc_status nc_bc_flags(nc_ctx* ctx, unsigned char* flags_host);

/* Optional element heat source s_e (Sec. 2, the s0 of the paper on the subdomain
 * omega), device array [E] of doubles copied into the context; NULL clears it.
 * Synchronous with respect to the given stream. */
nc_status nc_set_source(nc_ctx* ctx, const double* source_e, void* stream);

/* x_inout[D] := x_D: the Dirichlet values of the boundary conditions (Sec. 6.1:
 * zero velocity on walls, zero normal velocity on symmetry planes, T = 0 on the
 * cold walls, the prescribed patch temperature, p = 0 at a pinned node); other
 * entries are left unchanged.  x_inout: [5][Nn] DEVICE, double (NC_FP64) or
 * float (NC_FP32), owned by the caller.  Asynchronous on stream. */
nc_status nc_impose_dirichlet(nc_ctx* ctx, void* x_inout, int prec, void* stream);

/* Residual R(x, gamma) of the stabilised weak form (Sec. 4; App. B) plus the
 * patch flux term, Dirichlet rows x - x_D.  x, r: [5][Nn]; gamma: [E] with
 * gamma = 1 fluid, 0 solid (Sec. 3.1). */
nc_status nc_residual(nc_ctx* ctx, const void* x, const void* gamma, void* r, int prec,
                      void* stream);

/* Jv = J(x, gamma) v, the consistent Jacobian including the variation of the
 * stabilisation parameters with the velocity (App. B, dtau/du_e), matrix-free. */
nc_status nc_jvp(nc_ctx* ctx, const void* x, const void* gamma, const void* v, void* Jv,
                 int prec, void* stream);

/* JTw = J(x, gamma)^T w (the adjoint operator of Sec. 3.2), matrix-free. */
nc_status nc_jtvp(nc_ctx* ctx, const void* x, const void* gamma, const void* w, void* JTw,
                  int prec, void* stream);

/* Linearised products (FP64).  nc_linearize stores, for the state x and design
 * gamma, the state-only part of every quadrature point (velocity, velocity
 * gradient, temperature gradient and the strong residuals) and each element's
 * stabilisation parameters; nc_jvp_lin / nc_jtvp_lin then give the same J v and
 * J^T w as nc_jvp / nc_jtvp at that state without re-interpolating it -- the
 * products a Krylov solve applies many times at one state.  x and gamma are not
 * copied: they must stay unchanged while the linearisation is used.  The store
 * (about 1.2 KB per element) is allocated at the first call.  NC_ERR_ARG if
 * nc_jvp_lin / nc_jtvp_lin come before any nc_linearize. */
nc_status nc_linearize(nc_ctx* ctx, const double* x, const double* gamma, void* stream);
nc_status nc_jvp_lin(nc_ctx* ctx, const double* v, double* Jv, void* stream);
nc_status nc_jtvp_lin(nc_ctx* ctx, const double* w, double* JTw, void* stream);

/* d = diag(J(x, gamma)) (1 on Dirichlet rows): the Jacobi scaling of the
 * multigrid smoother (Sec. 5.2). */
nc_status nc_diag(nc_ctx* ctx, const void* x, const void* gamma, void* d, int prec,
                  void* stream);

/* Assembled Jacobian (the alternative to the matrix-free products): S receives
 * J(x, gamma) as a 27-point stencil of 5 x 5 blocks,
 *   S[((o*5 + f)*5 + g)*Nn + n] = dR(n, f) / dx(n + offset o, g),
 *   o = (dx+1) + 3 (dy+1) + 9 (dz+1), dx, dy, dz in {-1, 0, 1},
 * with entries reaching outside the grid 0, Dirichlet rows identity and
 * Dirichlet columns 0 (the same blockdiag(J_II, I) as nc_jvp).  S: DEVICE,
 * 675 Nn values of the precision prec, owned by the caller (5.4 KB per node in
 * FP64).  Built from the element Jacobians: 40 element products with unit
 * directions, each summed into S per node in a fixed order (deterministic); FP64
 * first stores the linearisation (as nc_linearize, in a context-owned store
 * allocated at the first call) and forms the columns from it with the unit
 * direction written out.  x and gamma as for nc_jvp. */
nc_status nc_assemble(nc_ctx* ctx, const void* x, const void* gamma, void* S, int prec,
                      void* stream);

/* out = S v, or S^T v with transpose, for a stencil S from nc_assemble (one thread
 * per node, neighbours in a fixed order).  v, out: [5][Nn] of the precision prec. */
nc_status nc_stencil_apply(nc_ctx* ctx, const void* S, const void* v, void* out, int transpose,
                           int prec, void* stream);

/* Objective.  With patch_mode NC_PATCH_NONE and an element source set
 * (nc_set_source): the thermal compliance of Sec. 3.2, f = int_omega s T dV.
 * Otherwise: the mean temperature of the bottom patch,
 * Phi = (1/|Gamma_p|) int T dA (the patch analogue of the same objective).
 * FP64 only.  phi_host receives the value (the call synchronises the stream);
 * dphidx, if not NULL, receives the gradient with respect to x as [5][Nn]. */
nc_status nc_objective(nc_ctx* ctx, const double* x, double* phi_host, double* dphidx,
                       void* stream);

/* Design sensitivities dPhi/dgamma_e = lambda^T dR/dgamma_e (Sec. 3.2, with
 * dtau/dgamma_e of App. B and dtau_T/dK_e), Dirichlet rows excluded, for the
 * adjoint lambda of J^T lambda = -dPhi/dx.  Output [E].  FP64 only. */
nc_status nc_sensitivity(nc_ctx* ctx, const double* x, const double* gamma,
                         const double* lambda, double* dphidgamma, void* stream);

/* Allocation-free J v.  The paper has no counterpart: this is a library
 * convenience for callers that may not allocate device memory -- an application
 * whose own memory pool has reserved the device and forbids other cudaMalloc
 * calls, a plug-in that must not make allocations its host does not track, or a
 * latency-bound loop that cannot afford the synchronisation cudaMalloc/cudaFree
 * may cause.  It computes the same product as nc_jvp (Dirichlet handling
 * included, no element source) without a context: the caller passes the
 * parameters, boundary conditions, inputs and output (device pointers, same
 * layouts and prec as nc_jvp), and the scratch is a fixed device array of
 * NC_STATIC_SCRATCH_BYTES inside the library, held by every GPU that loads it
 * until the process exits.  The problem must fit: round_up(Nn, 256) +
 * 40 * round_up(E, 32) * sizeof(element) <= NC_STATIC_SCRATCH_BYTES (about
 * 200,000 elements in FP64, 400,000 in FP32), else NC_ERR_SIZE and nothing is
 * launched.  The first call on
 * a device looks the array's device address up (once per device, with that
 * device current); make that first call before any stream capture.  The array
 * keeps the last call's contents; nothing in it needs to start at zero.  All
 * calls share it, so calls whose work can overlap on the GPU (different streams
 * or threads without ordering) race and must be serialised by the caller.
 * Errors: NC_ERR_ARG (a NULL pointer, or parameters or boundary conditions that
 * nc_setup would reject: sizes, coefficients, face conditions, patch mode, pinned
 * node), NC_ERR_SIZE, NC_ERR_CUDA. */
#define NC_STATIC_SCRATCH_BYTES (64ull << 20)
nc_status nc_jvp_static(const nc_params* prm, const nc_bcs* bcs, const void* x,
                        const void* gamma, const void* v, void* Jv, int prec, void* stream);

/* ALU throughput probe (a measurement helper; the paper has no counterpart).
 * The element operators are bound by the FP32 / FP64 pipes, so their roofline
 * is an arithmetic peak; this call measures what dependent FMA chains reach:
 * `blocks` blocks of 256 threads, each thread 8 independent chains of `iters`
 * fused multiply-adds (iters a positive multiple of 16), in double (NC_FP64) or
 * float (NC_FP32).  That is 16 * iters * blocks * 256 flop; time it with events
 * on `stream`.  out: DEVICE, blocks * 256 values of the precision, receives each
 * thread's chain sum.  Asynchronous.  NC_ERR_ARG for invalid arguments. */
nc_status nc_fma_probe(int prec, int blocks, long long iters, void* out, void* stream);

/* PDE (Helmholtz) density filter (Sec. 3.2; [Lazarov & Sigmund 2011]; the paper
 * uses radius = 2.5 h, Sec. 6.3-6.4): solves -r^2 lap(rho~) + rho~ = rho with
 * zero normal derivative on the boundary, r = radius / (2 sqrt 3), trilinear
 * nodal rho~ and element-constant rho, and returns the element means
 * gamma_f[e] of rho~ (element arrays [E], FP64, device).  The map rho -> gamma_f
 * is symmetric, so the same call applied to dPhi/dgamma_f gives dPhi/drho (the
 * chain rule of the filtered design).  Conjugate gradients with Jacobi
 * preconditioning to a relative residual of 1e-13; workspace (6 node vectors)
 * is allocated at the first call.  Synchronous.  NC_ERR_NAN for a non-finite
 * design, NC_ERR_MAXIT if CG does not converge in 1000 iterations. */
nc_status nc_filter(nc_ctx* ctx, const double* rho, double* gamma_f, double radius, void* stream);

/* Solver options.  rtol_newton: stop when ||R|| <= max(rtol_newton ||R_0||,
 * atol_newton) (Sec. 5.1 uses a relative tolerance);
 * rtol_lin: FGMRES relative tolerance per linear solve (Sec. 5.2), loosened inside
 * Newton to 0.01 of the Newton target divided by the current ||R|| when that is
 * larger (the last step near the target); max_newton,
 * max_lin (total FGMRES iterations per linear solve), restart (FGMRES restart,
 * <= 64); mg_levels: multigrid levels to use (0 = all); smooth_its: Jacobi-GMRES
 * smoothing iterations per pre/post step; coarse_its: Jacobi-GMRES iterations on
 * the coarsest level when it has more than 1000 unknowns (smaller coarsest levels
 * are solved with a dense inverse formed once per linearisation); mixed: 1 = Jacobian products, smoother and coarse levels
 * in FP32 inside FP64 Newton / refinement, 0 = everything FP64; ramp_steps: on
 * Newton failure (or stagnation) from the given start, continue in the buoyancy
 * from Gr / 10^ramp_steps up to Gr, each stage warm-started from the last, with
 * the step in log Gr halved after a failed stage and grown after a converged
 * one (0 = no ramping; the paper ramps the heat load, Sec. 5.1). */
typedef struct {
  double rtol_newton, rtol_lin;
  int max_newton, max_lin, restart;
  int mg_levels, smooth_its, coarse_its;
  int mixed;
  int ramp_steps;
  double atol_newton;  /* also stop when ||R|| <= atol_newton (default 0) */
  int galerkin;        /* 1: coarse-level operators are the Galerkin products P^T A P of the
                          level above (the paper's choice, Sec. 5.2), built by probing once
                          per linearisation and applied as 27-point block stencils; 0
                          (default): rediscretised at the injected state and averaged design */
  int assembled;       /* 1: every rediscretised level operator (level 0 included) is assembled
                          once per linearisation into a 27-point block stencil (as nc_assemble)
                          and applied as such; pays off in FP64 (mixed = 0), where an assembled
                          product costs about 0.4 of a matrix-free one and the assembly about
                          20 products; 0 (default): matrix-free */
  double rtol_adjoint; /* nc_adjoint_solve stops when ||rhs - J^T lambda|| <= rtol_adjoint ||rhs||
                          (default 1e-10; nc_newton_solve ignores it).  A residual bounds the
                          solution error only through the conditioning of J, so the adjoint
                          is solved 100 times tighter than the state's default 1e-8: the
                          mixed and FP64 sensitivities then agree to about 1e-9 */
  int adjoint_start;   /* nc_adjoint_solve's initial guess: 0 (default) lambda = 0; 1 the values
                          in lambda_inout on entry (e.g. the previous design iteration's adjoint,
                          as the state solve starts from the previous state, Sec. 5.1) */
} nc_solve_opts;

/* Per-solve report (Sec. 6.2 reports Newton and linear iteration counts). */
typedef struct {
  int newton_its, lin_its_total, status;
  double res0, res_final, seconds;
  double res_hist[64];
} nc_solve_info;

/* Fill opts with defaults (rtol_newton 1e-8, rtol_lin 1e-5, max_newton 30,
 * max_lin 200, restart 30, all levels, smooth_its 6, coarse_its 30, mixed 1,
 * ramp_steps 0, atol_newton 0, galerkin 0, assembled 0, rtol_adjoint 1e-10,
 * adjoint_start 0). */
void nc_default_opts(nc_solve_opts* opts);

/* Damped Newton (Sec. 5.1) on R(x, gamma) = 0 from x_inout (Dirichlet values
 * imposed first), step length from the quadratic fit of ||R|| at 0, 1/2 and 1
 * of the Newton step; each linear system by FGMRES preconditioned with a
 * geometric multigrid V-cycle whose smoother is Jacobi-preconditioned GMRES
 * (Sec. 5.2).  x_inout: [5][Nn] FP64, gamma: [E] FP64.  info may be NULL.
 * Synchronous. */
nc_status nc_newton_solve(nc_ctx* ctx, const double* gamma, double* x_inout,
                          const nc_solve_opts* opts, nc_solve_info* info, void* stream);

/* One orthogonalisation step of the FGMRES Arnoldi process (Sec. 5.2), the
 * same routine nc_newton_solve and nc_adjoint_solve run every iteration:
 * classical Gram-Schmidt applied twice against the k orthonormal columns
 * V_i = V + i*ldv (i < k), each of length n,
 *   h1 = V^T w,  w1 = w - V h1,  h2 = V^T w1,  w = (w1 - V h2) / nu,
 * with nu = ||w1 - V h2||, taken as sqrt(||w1||^2 - ||h2||^2) from the second
 * multi-dot (V orthonormal).  h_host receives k + 1 values: h1 + h2 (the new
 * Hessenberg column), then nu.  V and w: DEVICE arrays of double (NC_FP64) or
 * float (NC_FP32); the coefficients are double either way.  ldv >= n; columns
 * whose start is 16-byte aligned (ldv a multiple of 4 floats / 2 doubles and
 * an aligned V) take the 16-byte packet path.  A vanishing nu leaves w = w1 - V h2
 * unscaled.  Uses ctx's reduction scratch only (any context will do).
 * Synchronous.  NC_ERR_ARG if n < 1, k < 1, k > 64, ldv < n or a pointer is
 * NULL; NC_ERR_NAN if a coefficient is not finite. */
nc_status nc_arnoldi_orth(nc_ctx* ctx, long long n, int k, const void* V, long long ldv,
                          void* w, double* h_host, int prec, void* stream);

/* ---- design update (Sec. 3.2: minimise f subject to the volume constraint
 * g(gamma) = int_{Omega_d} (1 - gamma) dV <= v_f |Omega_d|, 0 <= gamma <= 1, by the
 * method of moving asymptotes [Svanberg 1987]).  Variables are element values
 * [n]; `active` (DEVICE, n bytes, may be NULL = all active) marks the design
 * variables: inactive ones take no part in the constraint and are never
 * changed by the update. */

/* Normalised volume constraint of a design gamma [n] (DEVICE, double):
 *   g = sum_active (1 - gamma_e) / (vf * n_active) - 1  (<= 0 when satisfied),
 * written to *g_host; dgdgamma (DEVICE [n], may be NULL) receives its gradient,
 * -1/(vf n_active) on active entries and 0 elsewhere (uniform elements, so the
 * integral is the element sum times h^3).  Synchronous.  NC_ERR_ARG for n < 1,
 * vf <= 0 or no active variable. */
nc_status nc_volume(nc_ctx* ctx, long long n, const double* gamma, const unsigned char* active,
                    double vf, double* g_host, double* dgdgamma, void* stream);

/* MMA options: move limit as a fraction of xmax - xmin, the box bounds, and a
 * positive factor applied to the objective gradient df0 (its scaling). */
typedef struct {
  double move;
  double xmin, xmax;
  double df0_scale;
} nc_mma_opts;

/* Fill opts with defaults (move 0.2, xmin 0, xmax 1, df0_scale 1). */
void nc_default_mma_opts(nc_mma_opts* opts);

/* out = min(max(in, lo), hi) on active entries and fixed (or 0 when fixed is
 * NULL) on the others: the physical design from the filtered variables with the
 * passive elements reset, or a gradient restricted to the design variables
 * (lo = -inf, hi = +inf, fixed NULL).  All DEVICE [n] double; out may alias in. */
nc_status nc_design_map(nc_ctx* ctx, long long n, const double* in, const unsigned char* active,
                        const double* fixed, double lo, double hi, double* out, void* stream);

/* One MMA iteration (iteration number iter, 0-based) for the objective with
 * gradient df0 (times opts->df0_scale) and one constraint of value f1 (<= 0
 * when satisfied) with gradient df1 (DEVICE [n] double each).  On entry x is the
 * current iterate, xold1 / xold2 the two before it and low / upp the previous
 * asymptotes (the three are ignored for iter < 2); on return x holds the new
 * iterate, xold1 / xold2 the shifted history and low / upp the asymptotes used
 * (all DEVICE [n] double, updated in place).  Asymptotes start at
 * x -/+ 0.5 (xmax - xmin) and then widen by 1.2 / narrow by 0.7 where a variable
 * moves monotonically / oscillates; move limits 0.1 of the way to the
 * asymptotes and `move` of the box; Svanberg's convex approximation of both
 * functions; the subproblem is solved through its dual, bisection on the
 * multiplier to floating-point resolution (the multiplier goes to
 * *lambda_host, and max_j |x_new - x| to *change_host; either may be NULL).
 * Synchronous.  NC_ERR_ARG for invalid sizes or options, NC_ERR_NAN for a
 * non-finite value. */
nc_status nc_mma_update(nc_ctx* ctx, long long n, int iter, double* x, double* xold1,
                        double* xold2, double* low, double* upp, const double* df0, double f1,
                        const double* df1, const unsigned char* active, const nc_mma_opts* opts,
                        double* lambda_host, double* change_host, void* stream);

/* Grid of multigrid level `level` (0 = the problem's grid; each level halves the
 * element counts while all of them stay even and at least 2): dims = {nx, ny, nz}. */
nc_status nc_level_dims(nc_ctx* ctx, int level, int* dims);

/* Apply the operator of multigrid level `level` as the solvers build it at the
 * linearisation point (x, gamma) (FP64 [5][Nn] and [E] of level 0): out = A_l v,
 * or A_l^T v with transpose.  Level 0 is the Jacobian J(x, gamma); coarser
 * levels are rediscretised at the injected state and the averaged design
 * (galerkin = 0) or the Galerkin products P^T A_{l-1} P of the trilinear
 * prolongation P (galerkin = 1, Sec. 5.2), with Dirichlet unknowns as identity
 * rows and removed columns.  v, out: DEVICE [5][Nn_l] of double (NC_FP64) or
 * float (NC_FP32, the mixed-precision hierarchy).  Builds the hierarchy's
 * linearisation first (the cost of a solver's linearisation).  Synchronous. */
nc_status nc_mg_apply(nc_ctx* ctx, int level, const double* x, const double* gamma, const void* v,
                      void* out, int prec, int transpose, int galerkin, void* stream);

/* Grid sequencing (nested iteration for a cold start): transfers between level
 * `level` (>= 1) of the hierarchy (nc_level_dims) and the finer level - 1.
 * nc_coarsen_elem: e_coarse[E_level] = mean of the eight children in
 * e_fine[E_{level-1}] (the design and source averaging of the hierarchy).
 * nc_prolong_state: x_fine[5][Nn_{level-1}] = trilinear interpolation of
 * x_coarse[5][Nn_level] (the multigrid prolongation), then the Dirichlet values
 * of the finer grid imposed.  A problem set up on level l's grid with the same
 * boundary conditions (and the pressure pin at node (i >> l, j >> l, k >> l))
 * is the level-l problem of the hierarchy.  FP64 DEVICE arrays, async. */
nc_status nc_coarsen_elem(nc_ctx* ctx, int level, const double* e_fine, double* e_coarse,
                          void* stream);
nc_status nc_prolong_state(nc_ctx* ctx, int level, const double* x_coarse, double* x_fine,
                           void* stream);

/* Adjoint solve J(x, gamma)^T lambda = rhs (Sec. 3.2) by FGMRES + multigrid on the
 * transposed operators, inside FP64 iterative refinement until
 * ||rhs - J^T lambda|| <= rtol_adjoint ||rhs|| (max_newton refinement sweeps at
 * most).  lambda_inout receives the solution; on entry it holds the initial
 * guess when opts->adjoint_start = 1 and is not read otherwise (start from 0).
 * info->res0 is ||rhs||, the refinement residuals go to info->res_hist (the
 * first one that of the initial guess).  The FP64 products J^T lambda of the
 * refinement come from an FP64 linearisation store of the finest grid: the FP64
 * solver's own (mixed = 0), or, with mixed = 1, one the context allocates at the
 * first adjoint solve (156 doubles per element, released by nc_destroy) when the
 * device keeps at least 8 GB free after it; otherwise they re-interpolate the
 * state.  All FP64 [5][Nn].  Synchronous. */
nc_status nc_adjoint_solve(nc_ctx* ctx, const double* x, const double* gamma,
                           const double* rhs, double* lambda_inout, const nc_solve_opts* opts,
                           nc_solve_info* info, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NC_H */
