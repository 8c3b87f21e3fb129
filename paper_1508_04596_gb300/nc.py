"""Python binding of libnc (argument marshalling only).

Every operation runs in the CUDA library ``libnc.so`` built from ``csrc/``; this
module checks tensor dtypes, devices and shapes, passes raw device pointers and
the current CUDA stream through the C ABI declared in ``include/nc.h``, and
turns status codes into exceptions.  There is no CPU fallback: importing this
module fails if the library has not been built.
"""
import ctypes
import os

import torch

from . import cavity, synth

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libnc.so is not built (run __graft_entry__.build() or "
                      "python -m paper_1508_04596_gb300.build); no CPU fallback exists")
lib = ctypes.CDLL(LIB_PATH)

NC_FP64, NC_FP32 = 0, 1
VEL_NOSLIP, VEL_FREE, VEL_SYMMETRY = 0, 1, 2
T_ADIABATIC, T_DIRICHLET = 0, 1
PATCH_NONE, PATCH_DIRICHLET, PATCH_FLUX = 0, 1, 2
STATUS = {0: "NC_OK", 1: "NC_ERR_ARG", 2: "NC_ERR_CUDA", 3: "NC_ERR_OOM", 4: "NC_ERR_NAN",
          5: "NC_ERR_MAXIT", 6: "NC_ERR_DIVERGED", 7: "NC_ERR_SIZE"}


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("Gr", ctypes.c_double), ("Pr", ctypes.c_double),
                ("alpha_max", ctypes.c_double), ("q_alpha", ctypes.c_double),
                ("q_f", ctypes.c_double), ("Ck", ctypes.c_double),
                ("g_dir", ctypes.c_double * 3)]


class BCs(ctypes.Structure):
    _fields_ = [("vel_bc", ctypes.c_int * 6), ("T_bc", ctypes.c_int * 6),
                ("T_val", ctypes.c_double * 6), ("patch", ctypes.c_double * 4),
                ("patch_mode", ctypes.c_int), ("patch_val", ctypes.c_double),
                ("p_pin", ctypes.c_longlong)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("rtol_newton", ctypes.c_double), ("rtol_lin", ctypes.c_double),
                ("max_newton", ctypes.c_int), ("max_lin", ctypes.c_int),
                ("restart", ctypes.c_int), ("mg_levels", ctypes.c_int),
                ("smooth_its", ctypes.c_int), ("coarse_its", ctypes.c_int),
                ("mixed", ctypes.c_int), ("ramp_steps", ctypes.c_int),
                ("atol_newton", ctypes.c_double), ("galerkin", ctypes.c_int),
                ("assembled", ctypes.c_int), ("rtol_adjoint", ctypes.c_double),
                ("adjoint_start", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("newton_its", ctypes.c_int), ("lin_its_total", ctypes.c_int),
                ("status", ctypes.c_int), ("res0", ctypes.c_double),
                ("res_final", ctypes.c_double), ("seconds", ctypes.c_double),
                ("res_hist", ctypes.c_double * 64)]

    def as_dict(self):
        k = min(self.newton_its + 1, 64)
        return dict(newton_its=self.newton_its, lin_its_total=self.lin_its_total,
                    status=STATUS.get(self.status, self.status), res0=self.res0,
                    res_final=self.res_final, seconds=self.seconds,
                    res_hist=list(self.res_hist[:k]))


class MmaOpts(ctypes.Structure):
    _fields_ = [("move", ctypes.c_double), ("xmin", ctypes.c_double), ("xmax", ctypes.c_double),
                ("df0_scale", ctypes.c_double)]


_vp = ctypes.c_void_p
_ctx = ctypes.c_void_p
_SIGS = {
    "nc_sizes": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]),
    "nc_setup": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.POINTER(BCs), ctypes.POINTER(_ctx)]),
    "nc_destroy": (None, [_ctx]),
    "nc_last_error": (ctypes.c_char_p, [_ctx]),
    "nc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "nc_bc_flags": (ctypes.c_int, [_ctx, _vp]),
    "nc_set_source": (ctypes.c_int, [_ctx, _vp, _vp]),
    "nc_impose_dirichlet": (ctypes.c_int, [_ctx, _vp, ctypes.c_int, _vp]),
    "nc_residual": (ctypes.c_int, [_ctx, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "nc_jvp": (ctypes.c_int, [_ctx, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "nc_jtvp": (ctypes.c_int, [_ctx, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "nc_diag": (ctypes.c_int, [_ctx, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "nc_objective": (ctypes.c_int, [_ctx, _vp, ctypes.POINTER(ctypes.c_double), _vp, _vp]),
    "nc_sensitivity": (ctypes.c_int, [_ctx, _vp, _vp, _vp, _vp, _vp]),
    "nc_default_opts": (None, [ctypes.POINTER(SolveOpts)]),
    "nc_filter": (ctypes.c_int, [_ctx, _vp, _vp, ctypes.c_double, _vp]),
    "nc_linearize": (ctypes.c_int, [_ctx, _vp, _vp, _vp]),
    "nc_assemble": (ctypes.c_int, [_ctx, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "nc_stencil_apply": (ctypes.c_int, [_ctx, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp]),
    "nc_jvp_lin": (ctypes.c_int, [_ctx, _vp, _vp, _vp]),
    "nc_jtvp_lin": (ctypes.c_int, [_ctx, _vp, _vp, _vp]),
    "nc_newton_solve": (ctypes.c_int, [_ctx, _vp, _vp, ctypes.POINTER(SolveOpts),
                                       ctypes.POINTER(SolveInfo), _vp]),
    "nc_adjoint_solve": (ctypes.c_int, [_ctx, _vp, _vp, _vp, _vp, ctypes.POINTER(SolveOpts),
                                        ctypes.POINTER(SolveInfo), _vp]),
    "nc_arnoldi_orth": (ctypes.c_int, [_ctx, ctypes.c_longlong, ctypes.c_int, _vp,
                                       ctypes.c_longlong, _vp, ctypes.POINTER(ctypes.c_double),
                                       ctypes.c_int, _vp]),
    "nc_level_dims": (ctypes.c_int, [_ctx, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "nc_coarsen_elem": (ctypes.c_int, [_ctx, ctypes.c_int, _vp, _vp, _vp]),
    "nc_prolong_state": (ctypes.c_int, [_ctx, ctypes.c_int, _vp, _vp, _vp]),
    "nc_mg_apply": (ctypes.c_int, [_ctx, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, _vp]),
    "nc_volume": (ctypes.c_int, [_ctx, ctypes.c_longlong, _vp, _vp, ctypes.c_double,
                                 ctypes.POINTER(ctypes.c_double), _vp, _vp]),
    "nc_default_mma_opts": (None, [ctypes.POINTER(MmaOpts)]),
    "nc_design_map": (ctypes.c_int, [_ctx, ctypes.c_longlong, _vp, _vp, _vp, ctypes.c_double,
                                     ctypes.c_double, _vp, _vp]),
    "nc_mma_update": (ctypes.c_int, [_ctx, ctypes.c_longlong, ctypes.c_int, _vp, _vp, _vp, _vp,
                                     _vp, _vp, ctypes.c_double, _vp, _vp,
                                     ctypes.POINTER(MmaOpts), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class NCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


def default_opts(**kw):
    o = SolveOpts()
    lib.nc_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def cavity_bcs(patch_mode=PATCH_DIRICHLET, patch_val=1.0, patch=(1 / 3, 2 / 3, 1 / 3, 2 / 3)):
    """Heated-base cavity: no-slip walls and bottom, traction-free top at T = 0,
    side walls at T = 0, bottom adiabatic outside a central patch that is held
    at T = patch_val or heated by the inward flux patch_val."""
    b = BCs()
    b.vel_bc[:] = [VEL_NOSLIP] * 5 + [VEL_FREE]
    b.T_bc[:] = [T_DIRICHLET] * 4 + [T_ADIABATIC, T_DIRICHLET]
    b.T_val[:] = [0.0] * 6
    b.patch[:] = list(patch)
    b.patch_mode = patch_mode
    b.patch_val = patch_val
    b.p_pin = -1
    return b


def quarter_bcs(nx, ny, nz):
    """The paper's quarter of a closed cavity (Sec. 6.1): symmetry planes on the
    +x and +y faces, no-slip elsewhere, cold (T = 0) outer vertical walls and
    top, insulated bottom; the pressure is pinned at the top outer corner node."""
    b = BCs()
    b.vel_bc[:] = [VEL_NOSLIP, VEL_SYMMETRY, VEL_NOSLIP, VEL_SYMMETRY, VEL_NOSLIP, VEL_NOSLIP]
    b.T_bc[:] = [T_DIRICHLET, T_ADIABATIC, T_DIRICHLET, T_ADIABATIC, T_ADIABATIC, T_DIRICHLET]
    b.T_val[:] = [0.0] * 6
    b.patch[:] = [0.0, 0.0, 0.0, 0.0]
    b.patch_mode = PATCH_NONE
    b.patch_val = 0.0
    b.p_pin = (nx + 1) * (ny + 1) * nz  # node (0, 0, nz)
    return b


def make_params(nx, ny, nz, h, Gr, Pr, alpha_max=1e4, q_alpha=1.0, q_f=1.0, Ck=0.1,
                g_dir=(0.0, 0.0, -1.0)):
    p = Params()
    p.nx, p.ny, p.nz, p.h = nx, ny, nz, h
    p.Gr, p.Pr = Gr, Pr
    p.alpha_max, p.q_alpha, p.q_f, p.Ck = alpha_max, q_alpha, q_f, Ck
    p.g_dir[:] = list(g_dir)
    return p


def mv_ld(n):
    """Column stride the solvers use for multivectors of length n (a multiple of
    64 elements, so that every column starts on a 256-byte boundary)."""
    return (n + 63) // 64 * 64


def coarse_pin(pin, fine_xy, coarse_xy):
    """Node index of a pressure pin on the next coarser grid: fine node (i, j, k)
    -> coarse node (i >> 1, j >> 1, k >> 1), as the multigrid hierarchy places it
    (-1, no pin, stays -1).  fine_xy / coarse_xy: element counts (nx, ny)."""
    if pin < 0:
        return pin
    nx1, ny1 = fine_xy[0] + 1, fine_xy[1] + 1
    i, j, k = pin % nx1, (pin // nx1) % ny1, pin // (nx1 * ny1)
    return (i >> 1) + (coarse_xy[0] + 1) * ((j >> 1) + (coarse_xy[1] + 1) * (k >> 1))


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)


class Problem:
    """A discrete problem on the current CUDA device (owns an nc_ctx)."""

    def __init__(self, params, bcs):
        self.params, self.bcs = params, bcs
        self.source = None
        ctx = _ctx()
        st = lib.nc_setup(ctypes.byref(params), ctypes.byref(bcs), ctypes.byref(ctx))
        if st != 0:
            raise NCError(st, "nc_setup failed")
        self.ctx = ctx
        nn, ne, nd = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        lib.nc_sizes(ctypes.byref(params), ctypes.byref(nn), ctypes.byref(ne), ctypes.byref(nd))
        self.Nn, self.E, self.ndof = nn.value, ne.value, nd.value

    @classmethod
    def from_workload(cls, name, **over):
        cfg = dict(synth.WORKLOADS[name])
        cfg.update(over)
        mat = synth.material(cfg)
        mat.update({k: over[k] for k in ("alpha_max", "q_alpha", "q_f", "Ck") if k in over})
        p = make_params(cfg["nx"], cfg["ny"], cfg["nz"], cfg["h"], cfg["Gr"], cfg["Pr"], **mat)
        if cfg.get("bcs") == "quarter":
            prob = cls(p, quarter_bcs(cfg["nx"], cfg["ny"], cfg["nz"]))
            s_e = cavity.source(cfg["nx"], cfg["ny"], cfg["nz"], cfg["h"], True)
            prob.set_source(torch.tensor(s_e, dtype=torch.float64, device="cuda"))
            return prob
        mode = PATCH_FLUX if cfg["patch"] == "flux" else PATCH_DIRICHLET
        return cls(p, cavity_bcs(mode, 1.0))

    def close(self):
        if getattr(self, "ctx", None):
            lib.nc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _chk(self, st):
        if st != 0:
            raise NCError(st, lib.nc_last_error(self.ctx).decode())

    def _vec(self, t, dtype, n, name):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dtype
                and t.is_contiguous() and t.numel() == n):
            raise ValueError("%s must be a contiguous CUDA %s tensor with %d elements" % (name, dtype, n))
        return ctypes.c_void_p(t.data_ptr())

    @staticmethod
    def _prec(x):
        return NC_FP64 if x.dtype == torch.float64 else NC_FP32

    # ---- operators -------------------------------------------------------
    def residual(self, x, gam, out=None, stream=None):
        out = torch.empty_like(x) if out is None else out
        dt = x.dtype
        self._chk(lib.nc_residual(self.ctx, self._vec(x, dt, self.ndof, "x"),
                                  self._vec(gam, dt, self.E, "gamma"),
                                  self._vec(out, dt, self.ndof, "r"), self._prec(x), _stream(stream)))
        return out

    def jvp(self, x, gam, v, out=None, stream=None):
        out = torch.empty_like(x) if out is None else out
        dt = x.dtype
        self._chk(lib.nc_jvp(self.ctx, self._vec(x, dt, self.ndof, "x"),
                             self._vec(gam, dt, self.E, "gamma"), self._vec(v, dt, self.ndof, "v"),
                             self._vec(out, dt, self.ndof, "Jv"), self._prec(x), _stream(stream)))
        return out

    def jtvp(self, x, gam, w, out=None, stream=None):
        out = torch.empty_like(x) if out is None else out
        dt = x.dtype
        self._chk(lib.nc_jtvp(self.ctx, self._vec(x, dt, self.ndof, "x"),
                              self._vec(gam, dt, self.E, "gamma"), self._vec(w, dt, self.ndof, "w"),
                              self._vec(out, dt, self.ndof, "JTw"), self._prec(x), _stream(stream)))
        return out

    STENCIL_VALUES = 675

    def assemble(self, x, gam, S=None, stream=None):
        """The Jacobian J(x, gamma) assembled as a 27-point stencil of 5 x 5 blocks:
        S[((o*5 + f)*5 + g)*Nn + n] couples (n, f) to (n + offset o, g), with
        o = (dx+1) + 3 (dy+1) + 9 (dz+1); 675 Nn values of x's dtype."""
        dt = x.dtype
        n = self.STENCIL_VALUES * self.Nn
        S = torch.empty(n, dtype=dt, device=x.device) if S is None else S
        self._chk(lib.nc_assemble(self.ctx, self._vec(x, dt, self.ndof, "x"),
                                  self._vec(gam, dt, self.E, "gamma"), self._vec(S, dt, n, "S"),
                                  self._prec(x), _stream(stream)))
        return S

    def stencil_apply(self, S, v, out=None, transpose=False, stream=None):
        """out = S v (or S^T v) for a stencil from assemble()."""
        dt = v.dtype
        out = torch.empty_like(v) if out is None else out
        self._chk(lib.nc_stencil_apply(self.ctx, self._vec(S, dt, self.STENCIL_VALUES * self.Nn, "S"),
                                       self._vec(v, dt, self.ndof, "v"),
                                       self._vec(out, dt, self.ndof, "out"), int(transpose),
                                       self._prec(v), _stream(stream)))
        return out

    def arnoldi_orth(self, V, w, k, ldv, stream=None):
        """One FGMRES orthogonalisation step (classical Gram-Schmidt twice) of w
        against the k orthonormal columns V[i*ldv : i*ldv + n], n = w.numel();
        w is overwritten by the new unit basis vector.  Returns the k + 1
        coefficients (the Hessenberg column, then the norm) as a list."""
        n = w.numel()
        if not (isinstance(V, torch.Tensor) and V.is_cuda and V.dtype == w.dtype
                and V.is_contiguous() and V.numel() >= (k - 1) * ldv + n):
            raise ValueError("V must be a contiguous CUDA tensor of w's dtype holding k columns")
        self._vec(w, w.dtype, n, "w")
        h = (ctypes.c_double * (k + 1))()
        self._chk(lib.nc_arnoldi_orth(self.ctx, n, k, ctypes.c_void_p(V.data_ptr()), ldv,
                                      ctypes.c_void_p(w.data_ptr()), h, self._prec(w),
                                      _stream(stream)))
        return list(h)

    # ---- multigrid levels (Sec. 5.2) ---------------------------------------
    def level_dims(self, level):
        d = (ctypes.c_int * 3)()
        self._chk(lib.nc_level_dims(self.ctx, level, d))
        return tuple(d)

    def mg_apply(self, level, x, gam, v, out=None, transpose=False, galerkin=False, stream=None):
        """out = A_l v (or A_l^T v) with the multigrid level-l operator built at
        (x, gamma); v and out hold 5 (nx_l+1)(ny_l+1)(nz_l+1) values."""
        nx, ny, nz = self.level_dims(level)
        n = 5 * (nx + 1) * (ny + 1) * (nz + 1)
        out = torch.empty_like(v) if out is None else out
        self._vec(v, v.dtype, n, "v")
        self._vec(out, v.dtype, n, "out")
        self._chk(lib.nc_mg_apply(self.ctx, level, self._vec(x, torch.float64, self.ndof, "x"),
                                  self._vec(gam, torch.float64, self.E, "gamma"),
                                  ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  self._prec(v), int(transpose), int(galerkin), _stream(stream)))
        return out

    # ---- grid sequencing ----------------------------------------------------
    def coarse_problem(self):
        """The problem on the next coarser grid of the multigrid hierarchy (element
        counts halved, h doubled, the same boundary conditions, the pressure pin
        at the coarse node (i >> 1, j >> 1, k >> 1), the element source averaged
        over the children), or None when the grid does not halve."""
        d = (ctypes.c_int * 3)()
        if lib.nc_level_dims(self.ctx, 1, d) != 0:
            return None
        p = Params.from_buffer_copy(self.params)
        p.nx, p.ny, p.nz, p.h = d[0], d[1], d[2], 2.0 * self.params.h
        b = BCs.from_buffer_copy(self.bcs)
        b.p_pin = coarse_pin(b.p_pin, (self.params.nx, self.params.ny), (d[0], d[1]))
        c = Problem(p, b)
        if self.source is not None:
            c.set_source(self.coarsen(self.source))
        return c

    def coarsen(self, e, stream=None):
        """Element field on the next coarser grid: the mean of each element's 8 children."""
        d = (ctypes.c_int * 3)()
        self._chk(lib.nc_level_dims(self.ctx, 1, d))
        out = torch.empty(d[0] * d[1] * d[2], dtype=torch.float64, device=e.device)
        self._chk(lib.nc_coarsen_elem(self.ctx, 1, self._vec(e, torch.float64, self.E, "e"),
                                      ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def prolong(self, xc, stream=None):
        """State on this grid from the next coarser grid's (trilinear, Dirichlet
        values imposed)."""
        d = (ctypes.c_int * 3)()
        self._chk(lib.nc_level_dims(self.ctx, 1, d))
        nc_ = 5 * (d[0] + 1) * (d[1] + 1) * (d[2] + 1)
        out = torch.empty(self.ndof, dtype=torch.float64, device=xc.device)
        self._chk(lib.nc_prolong_state(self.ctx, 1, self._vec(xc, torch.float64, nc_, "x_coarse"),
                                       ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def newton_solve_sequenced(self, gam, x, opts=None, coarse_opts=None, stream=None, check=True):
        """Cold start by grid sequencing (nested iteration): the state is solved on
        every coarser grid of the hierarchy first, coarsest first, and each
        solution, prolonged, starts the solve on the next finer grid; x receives
        the solution on this grid.  coarse_opts (default opts) apply to the
        coarser solves.  Returns (x, info) of the final solve, with
        info["levels"] reporting the coarser ones (coarsest first).  A coarser
        solve that does not converge is not prolonged: the next finer grid then
        starts from zero, and its entry in info["levels"] has prolonged=False."""
        chain, gams = [self], [gam]
        while True:
            c = chain[-1].coarse_problem()
            if c is None:
                break
            gams.append(chain[-1].coarsen(gams[-1], stream))
            chain.append(c)
        xs = torch.zeros(chain[-1].ndof, dtype=torch.float64, device=x.device)
        levels = []
        for k in range(len(chain) - 1, 0, -1):
            _, inf = chain[k].newton_solve(gams[k], xs, coarse_opts or opts, stream, check=False)
            pk = chain[k].params
            ok = inf["status"] == "NC_OK"
            levels.append(dict(dims=(pk.nx, pk.ny, pk.nz), status=inf["status"],
                               newton_its=inf["newton_its"], lin_its=inf["lin_its_total"],
                               seconds=inf["seconds"], prolonged=ok))
            if ok:
                xs = chain[k - 1].prolong(xs, stream)
            else:  # a failed coarse state would only mislead the finer solve
                xs = torch.zeros(chain[k - 1].ndof, dtype=torch.float64, device=x.device)
            chain[k].close()  # free the coarser context before the finer solve
        x.copy_(xs)
        del xs
        _, info = self.newton_solve(gam, x, opts, stream, check)
        info["levels"] = levels
        return x, info

    # ---- design update (Sec. 3.2) ------------------------------------------
    def volume(self, gam, active=None, vf=0.05, grad=None, stream=None):
        """Normalised volume constraint g = sum_active (1 - gamma)/(vf n_active) - 1
        (Sec. 3.2) and, into grad if given, its gradient."""
        n = gam.numel()
        self._vec(gam, torch.float64, n, "gamma")
        if active is not None:
            self._vec(active, torch.uint8, n, "active")
        if grad is not None:
            self._vec(grad, torch.float64, n, "grad")
        g = ctypes.c_double()
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        self._chk(lib.nc_volume(self.ctx, n, p(gam), p(active), vf, ctypes.byref(g), p(grad),
                                _stream(stream)))
        return g.value

    def design_map(self, v, active=None, fixed=None, lo=-float("inf"), hi=float("inf"), out=None,
                   stream=None):
        """clamp(v, lo, hi) on active entries, fixed (or 0) elsewhere."""
        n = v.numel()
        out = torch.empty_like(v) if out is None else out
        self._vec(v, torch.float64, n, "v")
        self._vec(out, torch.float64, n, "out")
        if active is not None:
            self._vec(active, torch.uint8, n, "active")
        if fixed is not None:
            self._vec(fixed, torch.float64, n, "fixed")
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        self._chk(lib.nc_design_map(self.ctx, n, p(v), p(active), p(fixed), lo, hi, p(out),
                                    _stream(stream)))
        return out

    def mma_update(self, it, x, xold1, xold2, low, upp, df0, f1, df1, active=None,
                   move=0.2, xmin=0.0, xmax=1.0, df0_scale=1.0, stream=None):
        """One MMA iteration (Sec. 3.2, Svanberg 1987); x, xold1, xold2, low, upp
        are updated in place.  Returns (constraint multiplier, max |x_new - x|)."""
        n = x.numel()
        for t, nm in ((x, "x"), (xold1, "xold1"), (xold2, "xold2"), (low, "low"), (upp, "upp"),
                      (df0, "df0"), (df1, "df1")):
            self._vec(t, torch.float64, n, nm)
        if active is not None:
            self._vec(active, torch.uint8, n, "active")
        o = MmaOpts()
        lib.nc_default_mma_opts(ctypes.byref(o))
        o.move, o.xmin, o.xmax, o.df0_scale = move, xmin, xmax, df0_scale
        lam, chg = ctypes.c_double(), ctypes.c_double()
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
        self._chk(lib.nc_mma_update(self.ctx, n, it, p(x), p(xold1), p(xold2), p(low), p(upp),
                                    p(df0), float(f1), p(df1), p(active), ctypes.byref(o),
                                    ctypes.byref(lam), ctypes.byref(chg), _stream(stream)))
        return lam.value, chg.value

    def linearize(self, x, gam, stream=None):
        """Store the linearisation at (x, gamma) (FP64); x and gamma must stay
        unchanged while jvp_lin / jtvp_lin use it."""
        self._lin = (x, gam)  # keep the tensors alive
        self._chk(lib.nc_linearize(self.ctx, self._vec(x, torch.float64, self.ndof, "x"),
                                   self._vec(gam, torch.float64, self.E, "gamma"),
                                   _stream(stream)))

    def jvp_lin(self, v, out=None, stream=None):
        out = torch.empty_like(v) if out is None else out
        self._chk(lib.nc_jvp_lin(self.ctx, self._vec(v, torch.float64, self.ndof, "v"),
                                 self._vec(out, torch.float64, self.ndof, "Jv"), _stream(stream)))
        return out

    def jtvp_lin(self, w, out=None, stream=None):
        out = torch.empty_like(w) if out is None else out
        self._chk(lib.nc_jtvp_lin(self.ctx, self._vec(w, torch.float64, self.ndof, "w"),
                                  self._vec(out, torch.float64, self.ndof, "JTw"), _stream(stream)))
        return out

    def diag(self, x, gam, out=None, stream=None):
        out = torch.empty_like(x) if out is None else out
        dt = x.dtype
        self._chk(lib.nc_diag(self.ctx, self._vec(x, dt, self.ndof, "x"),
                              self._vec(gam, dt, self.E, "gamma"),
                              self._vec(out, dt, self.ndof, "d"), self._prec(x), _stream(stream)))
        return out

    def impose_dirichlet(self, x, stream=None):
        self._chk(lib.nc_impose_dirichlet(self.ctx, self._vec(x, x.dtype, self.ndof, "x"),
                                          self._prec(x), _stream(stream)))
        return x

    def bc_flags(self):
        import numpy as np
        out = np.zeros(self.Nn, dtype=np.uint8)
        self._chk(lib.nc_bc_flags(self.ctx, ctypes.c_void_p(out.ctypes.data)))
        return out

    def set_source(self, s_e, stream=None):
        p = None if s_e is None else self._vec(s_e, torch.float64, self.E, "source")
        self._chk(lib.nc_set_source(self.ctx, p, _stream(stream)))
        self.source = s_e

    def objective(self, x, want_grad=True, stream=None):
        phi = ctypes.c_double()
        g = torch.empty_like(x) if want_grad else None
        self._chk(lib.nc_objective(self.ctx, self._vec(x, torch.float64, self.ndof, "x"),
                                   ctypes.byref(phi),
                                   None if g is None else ctypes.c_void_p(g.data_ptr()),
                                   _stream(stream)))
        return phi.value, g

    def sensitivity(self, x, gam, lam, out=None, stream=None):
        out = torch.empty_like(gam) if out is None else out
        self._chk(lib.nc_sensitivity(self.ctx, self._vec(x, torch.float64, self.ndof, "x"),
                                     self._vec(gam, torch.float64, self.E, "gamma"),
                                     self._vec(lam, torch.float64, self.ndof, "lambda"),
                                     self._vec(out, torch.float64, self.E, "dphidgamma"),
                                     _stream(stream)))
        return out

    def filter(self, rho, radius=None, out=None, stream=None):
        """PDE density filter (Sec. 3.2); radius defaults to 2.5 h (Sec. 6.3).
        Symmetric: applied to dPhi/dgamma~ it returns dPhi/drho."""
        out = torch.empty_like(rho) if out is None else out
        R = 2.5 * self.params.h if radius is None else radius
        self._chk(lib.nc_filter(self.ctx, self._vec(rho, torch.float64, self.E, "rho"),
                                self._vec(out, torch.float64, self.E, "gamma_f"), R,
                                _stream(stream)))
        return out

    # ---- solvers ---------------------------------------------------------
    def newton_solve(self, gam, x, opts=None, stream=None, check=True):
        opts = default_opts() if opts is None else opts
        info = SolveInfo()
        st = lib.nc_newton_solve(self.ctx, self._vec(gam, torch.float64, self.E, "gamma"),
                                 self._vec(x, torch.float64, self.ndof, "x"), ctypes.byref(opts),
                                 ctypes.byref(info), _stream(stream))
        if check:
            self._chk(st)
        return x, info.as_dict()

    def adjoint_solve(self, x, gam, rhs, lam=None, opts=None, stream=None, check=True):
        """J^T lam = rhs.  lam (optional) receives the solution; with
        opts.adjoint_start = 1 its values on entry are the initial guess."""
        opts = default_opts() if opts is None else opts
        if lam is None:
            if opts.adjoint_start:
                raise ValueError("adjoint_start = 1 needs the initial guess in lam")
            lam = torch.empty_like(x)
        info = SolveInfo()
        st = lib.nc_adjoint_solve(self.ctx, self._vec(x, torch.float64, self.ndof, "x"),
                                  self._vec(gam, torch.float64, self.E, "gamma"),
                                  self._vec(rhs, torch.float64, self.ndof, "rhs"),
                                  self._vec(lam, torch.float64, self.ndof, "lambda"),
                                  ctypes.byref(opts), ctypes.byref(info), _stream(stream))
        if check:
            self._chk(st)
        return lam, info.as_dict()


class DensityFilter(torch.autograd.Function):
    """gamma~ = P rho, the PDE density filter (Sec. 3.2); P is symmetric, so the
    backward pass applies the same filter to the incoming gradient."""

    @staticmethod
    def forward(ctx, rho, prob, radius=None):
        ctx.prob, ctx.radius = prob, radius
        return prob.filter(rho.detach().contiguous(), radius)

    @staticmethod
    def backward(ctx, grad):
        return ctx.prob.filter(grad.contiguous(), ctx.radius), None, None


class PatchTemperature(torch.autograd.Function):
    """Phi(gamma) = mean patch temperature of the converged state (forward:
    Newton solve + objective); backward: adjoint solve J^T lambda = -dPhi/dx and
    the element sensitivities lambda^T dR/dgamma (Sec. 3.2, App. B)."""

    @staticmethod
    def forward(ctx, gam, prob, x0, opts):
        x = x0.detach().clone()
        prob.newton_solve(gam.detach(), x, opts)
        phi, dphi = prob.objective(x)
        ctx.prob, ctx.opts = prob, opts
        ctx.save_for_backward(gam.detach(), x, dphi)
        return torch.tensor(phi, dtype=torch.float64, device=gam.device)

    @staticmethod
    def backward(ctx, grad):
        gam, x, dphi = ctx.saved_tensors
        lam, _ = ctx.prob.adjoint_solve(x, gam, -dphi, opts=ctx.opts)
        sens = ctx.prob.sensitivity(x, gam, lam)
        return grad * sens, None, None, None
