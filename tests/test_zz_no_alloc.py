"""The allocation-free J v (nc_jvp_static) against the context-based nc_jvp and
against the oracle's assembled Jacobian.

nc_jvp_static exists for callers that may not allocate device memory (an
application whose memory pool owns the device, a plug-in whose host tracks every
allocation, a loop that cannot afford cudaMalloc's synchronisation); it keeps its
scratch in a fixed array inside the library.  This test calls it through the C
ABI twice in a row -- the second call reuses the scratch the first one left
behind -- and compares each result with nc_jvp on the same inputs, and with the
oracle's J v on two boundary-condition sets (the heated cavity with a patch held
at T = 1, and a set with symmetry planes, a pinned pressure node and a
flux-heated patch, which exercises every rule of the entry point's own
boundary-flag kernel), within the tolerances of the other parity tests.  It runs last in a collection so that a
failure here cannot hide another test's result.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_04596_gb300 import nc as ncmod
    f = ncmod.lib.nc_jvp_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(ncmod.Params), ctypes.POINTER(ncmod.BCs)] + [ctypes.c_void_p] * 4 \
        + [ctypes.c_int, ctypes.c_void_p]
    return ncmod


def call_static(nc, p, b, x, g, v, out, prec):
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return nc.lib.nc_jvp_static(ctypes.byref(p), ctypes.byref(b), ctypes.c_void_p(x.data_ptr()),
                                ctypes.c_void_p(g.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), prec, s)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_static_jvp_matches_context_jvp_twice(nc, prec):
    from paper_1508_04596_gb300 import synth
    nx, ny, nz = 24, 20, 16
    h = 1.0 / nx
    p = nc.make_params(nx, ny, nz, h, 1e4, 0.71, **synth.MATERIAL)
    b = nc.cavity_bcs(nc.PATCH_DIRICHLET, 1.0)
    prob = nc.Problem(p, b)
    dt, code, tol = ((torch.float64, nc.NC_FP64, 1e-12) if prec == "f64"
                     else (torch.float32, nc.NC_FP32, 2e-4))
    g = torch.tensor(synth.smoothed_random(nx, ny, nz, h, 7), dtype=dt, device="cuda")
    x = torch.tensor(synth.random_state(nx, ny, nz, 8, (0.5, 0.5, 0.5, 50.0, 1.0)).ravel(),
                     dtype=dt, device="cuda")
    prob.impose_dirichlet(x)
    rng = np.random.default_rng(9)
    for call in range(2):
        v = torch.tensor(rng.standard_normal(prob.ndof), dtype=dt, device="cuda")
        ref = prob.jvp(x, g, v)
        out = torch.full_like(x, float("nan"))
        assert call_static(nc, p, b, x, g, v, out, code) == 0
        torch.cuda.synchronize()
        err = (torch.linalg.norm((out - ref).double()) / torch.linalg.norm(ref.double())).item()
        assert err <= tol, (call, err)


def test_static_jvp_rejects_oversize(nc):
    from paper_1508_04596_gb300 import synth
    n = 80  # 512,000 elements: 40 * E * 8 bytes is far beyond the fixed scratch
    p = nc.make_params(n, n, n, 1.0 / n, 1e4, 0.71, **synth.MATERIAL)
    b = nc.cavity_bcs()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")  # never touched
    assert call_static(nc, p, b, t, t, t, t, nc.NC_FP64) == 7  # NC_ERR_SIZE
    assert nc.lib.nc_status_string(7).startswith(b"problem larger")


def _bc_sets(nc, nx, ny, nz):
    from oracle import grid as G
    cav = (nc.cavity_bcs(nc.PATCH_DIRICHLET, 1.0), G.BCs(patch_mode=G.PATCH_DIRICHLET))
    pin = 3 + (nx + 1) * (2 + (ny + 1) * nz)  # a node on the top face
    b = nc.BCs()
    b.vel_bc[:] = [nc.VEL_NOSLIP, nc.VEL_SYMMETRY, nc.VEL_SYMMETRY, nc.VEL_NOSLIP,
                   nc.VEL_NOSLIP, nc.VEL_FREE]
    b.T_bc[:] = [nc.T_DIRICHLET, nc.T_ADIABATIC, nc.T_ADIABATIC, nc.T_DIRICHLET,
                 nc.T_ADIABATIC, nc.T_DIRICHLET]
    b.T_val[:] = [0.0] * 6
    b.patch[:] = [1 / 3, 2 / 3, 1 / 3, 2 / 3]
    b.patch_mode, b.patch_val, b.p_pin = nc.PATCH_FLUX, 1.0, pin
    o = G.BCs(vel_bc=(G.NOSLIP, G.SYMMETRY, G.SYMMETRY, G.NOSLIP, G.NOSLIP, G.FREE),
              T_bc=(G.DIRICHLET, G.ADIABATIC, G.ADIABATIC, G.DIRICHLET, G.ADIABATIC, G.DIRICHLET),
              patch_mode=G.PATCH_FLUX, p_pin=pin)
    return {"cavity": cav, "symmetry_pin_flux": (b, o)}


@pytest.mark.parametrize("bcset", ["cavity", "symmetry_pin_flux"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_static_jvp_matches_oracle_twice(nc, prec, bcset):
    from paper_1508_04596_gb300 import synth
    from tests.helpers import oracle_problem, random_bc_state
    nx, ny, nz = 9, 7, 10
    h = 1.0 / nx
    b, ob = _bc_sets(nc, nx, ny, nz)[bcset]
    p = nc.make_params(nx, ny, nz, h, 1e4, 0.71, **synth.MATERIAL)
    prob, _ = oracle_problem(nx, ny, nz, h, 1e4, 0.71, bc=ob)
    gam = synth.smoothed_random(nx, ny, nz, h, 5)
    x = random_bc_state(prob, 6)
    J = prob.jacobian(x, gam)
    dt, code, tol = ((torch.float64, nc.NC_FP64, 1e-12) if prec == "f64"
                     else (torch.float32, nc.NC_FP32, 2e-4))
    xd = torch.tensor(x.ravel(), dtype=dt, device="cuda")
    gd = torch.tensor(gam, dtype=dt, device="cuda")
    rng = np.random.default_rng(10)
    for call in range(2):
        v = rng.standard_normal(prob.g.ndof)
        out = torch.full_like(xd, float("nan"))
        assert call_static(nc, p, b, xd, gd, torch.tensor(v, dtype=dt, device="cuda"), out,
                           code) == 0
        torch.cuda.synchronize()
        ref = J @ v
        err = float(np.linalg.norm(out.double().cpu().numpy() - ref) / np.linalg.norm(ref))
        assert err <= tol, (call, err)


def test_static_jvp_rejects_invalid_arguments(nc):
    """The checks of nc_setup: a patch mode out of range, a non-finite Gr, a
    negative alpha_max and a dimension too large to form its products are
    NC_ERR_ARG before anything is launched."""
    t = torch.zeros(1, dtype=torch.float64, device="cuda")  # never touched
    b = nc.cavity_bcs()
    b.patch_mode = 3
    assert call_static(nc, nc.make_params(4, 4, 4, 0.25, 1e3, 0.71), b, t, t, t, t,
                       nc.NC_FP64) == 1
    for p in (nc.make_params(4, 4, 4, 0.25, float("inf"), 0.71),
              nc.make_params(4, 4, 4, 0.25, 1e3, 0.71, alpha_max=-1.0),
              nc.make_params(2 ** 31 - 1, 4, 4, 0.25, 1e3, 0.71)):
        assert call_static(nc, p, nc.cavity_bcs(), t, t, t, t, nc.NC_FP64) == 1
