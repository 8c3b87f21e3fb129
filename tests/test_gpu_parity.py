"""GPU parity: libnc (through its C ABI) against the FP64 oracle on the same
seeded inputs.

Tolerances.  FP64: relative L2 <= 1e-12 for the residual, J v, J^T w, diag(J)
and the element sensitivities (random BC-consistent states, ||R|| = O(1)).
Integer work (boundary flags) is compared bit for bit.  FP32: the kernels round
every input to FP32 (relative 6e-8) and accumulate about 10^3 terms per output
in FP32, with cancellation between the pressure gradient and the buoyancy term
of up to two orders of magnitude; the bound used is relative L2 <= 2e-4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import grid as G  # noqa: E402
from oracle import solve as S  # noqa: E402
from paper_1508_04596_gb300 import synth  # noqa: E402
from tests.helpers import oracle_problem, random_bc_state, sampled_rows  # noqa: E402

TOL64 = 1e-12
TOL32 = 2e-4


@pytest.fixture(scope="module")
def nc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_04596_gb300 import nc as ncmod
    return ncmod


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a).ravel(), dtype=dtype, device="cuda")


def host(t, shape=None):
    a = t.detach().double().cpu().numpy()
    return a if shape is None else a.reshape(shape)


# grids: cfg-0 cube, ragged non-cubic, flux patch, and the degenerate grids of one
# element and of one element across
CASES = [
    dict(nx=12, ny=12, nz=12, Gr=1e3, patch="dirichlet", seed=0),
    dict(nx=5, ny=7, nz=6, Gr=1e4, patch="flux", seed=1),
    dict(nx=9, ny=4, nz=3, Gr=1e5, patch="dirichlet", seed=2),
    dict(nx=1, ny=1, nz=1, Gr=1e3, patch="dirichlet", seed=3),
    dict(nx=2, ny=1, nz=3, Gr=1e4, patch="flux", seed=4),
]


def make_pair(nc, c):
    h = 1.0 / c["nx"]
    prob, bc = oracle_problem(c["nx"], c["ny"], c["nz"], h, c["Gr"], 0.71, patch_mode=c["patch"])
    p = nc.make_params(c["nx"], c["ny"], c["nz"], h, c["Gr"], 0.71, **synth.MATERIAL)
    mode = nc.PATCH_FLUX if c["patch"] == "flux" else nc.PATCH_DIRICHLET
    gp = nc.Problem(p, nc.cavity_bcs(mode, 1.0))
    gam = synth.smoothed_random(c["nx"], c["ny"], c["nz"], h, c["seed"])
    x = random_bc_state(prob, 100 + c["seed"])
    return prob, bc, gp, gam, x


@pytest.mark.parametrize("c", CASES)
def test_bc_flags_bit_exact(nc, c):
    prob, bc, gp, gam, x = make_pair(nc, c)
    fl = gp.bc_flags()
    mask = np.zeros((5, prob.g.Nn), bool)
    for f in range(5):
        mask[f] = (fl >> f) & 1
    assert np.array_equal(mask, prob.dmask)


def test_bc_flags_symmetry_and_pin(nc):
    bc = G.BCs(vel_bc=(G.SYMMETRY, G.NOSLIP, G.NOSLIP, G.SYMMETRY, G.NOSLIP, G.NOSLIP),
               patch_mode=G.PATCH_FLUX, p_pin=7)
    prob, _ = oracle_problem(4, 6, 5, 0.25, 1e3, 0.71, bc=bc)
    b = nc.BCs()
    b.vel_bc[:] = [2, 0, 0, 2, 0, 0]
    b.T_bc[:] = [1, 1, 1, 1, 0, 1]
    b.T_val[:] = [0.0] * 6
    b.patch[:] = [1 / 3, 2 / 3, 1 / 3, 2 / 3]
    b.patch_mode, b.patch_val, b.p_pin = 2, 1.0, 7
    gp = nc.Problem(nc.make_params(4, 6, 5, 0.25, 1e3, 0.71), b)
    fl = gp.bc_flags()
    for f in range(5):
        assert np.array_equal(((fl >> f) & 1).astype(bool), prob.dmask[f])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_operators_interior_pin(nc, prec):
    """Pressure pinned at an interior node (the one Dirichlet node that can lie off
    the boundary): J v and J^T w against the oracle's Jacobian, and the residual."""
    nx, ny, nz = 36, 10, 9
    pin = 5 + (nx + 1) * (4 + (ny + 1) * 3)
    bc = G.BCs(patch_mode=G.PATCH_FLUX, p_pin=pin)
    prob, _ = oracle_problem(nx, ny, nz, 1.0 / nx, 1e4, 0.71, bc=bc)
    b = nc.cavity_bcs(nc.PATCH_FLUX, 1.0)
    b.p_pin = pin
    gp = nc.Problem(nc.make_params(nx, ny, nz, 1.0 / nx, 1e4, 0.71, **synth.MATERIAL), b)
    assert ((gp.bc_flags()[pin] >> 3) & 1) == 1
    gam = synth.smoothed_random(nx, ny, nz, 1.0 / nx, 31)
    x = random_bc_state(prob, 32)
    J = prob.jacobian(x, gam)
    dt, tol = (torch.float64, TOL64) if prec == "f64" else (torch.float32, TOL32)
    xd, gd = dev(x, dt), dev(gam, dt)
    v = np.random.default_rng(33).standard_normal(prob.g.ndof)
    vd = dev(v, dt)
    assert rel(host(gp.residual(xd, gd), (5, -1)), prob.residual(x, gam)) <= tol
    assert rel(host(gp.jvp(xd, gd, vd)), J @ v) <= tol
    assert rel(host(gp.jtvp(xd, gd, vd)), J.T @ v) <= tol


@pytest.mark.parametrize("c", CASES)
def test_residual_fp64(nc, c):
    prob, bc, gp, gam, x = make_pair(nc, c)
    R = gp.residual(dev(x), dev(gam))
    Ro = prob.residual(x, gam)
    assert np.linalg.norm(Ro) > 1e-3
    assert rel(host(R, Ro.shape), Ro) <= TOL64


@pytest.mark.parametrize("c", CASES)
def test_jvp_jtvp_diag_fp64(nc, c):
    prob, bc, gp, gam, x = make_pair(nc, c)
    J = prob.jacobian(x, gam)
    xd, gd = dev(x), dev(gam)
    rng = np.random.default_rng(c["seed"] + 7)
    for s in range(16 if c["nx"] == 12 else 4):
        v = rng.standard_normal(prob.g.ndof)
        Jv = gp.jvp(xd, gd, dev(v))
        assert rel(host(Jv), J @ v) <= TOL64
        JTw = gp.jtvp(xd, gd, dev(v))
        assert rel(host(JTw), J.T @ v) <= TOL64
    d = gp.diag(xd, gd)
    assert rel(host(d), J.diagonal()) <= TOL64


@pytest.mark.parametrize("c", CASES)
def test_linearised_products_fp64(nc, c):
    """nc_linearize + nc_jvp_lin / nc_jtvp_lin: the cached products equal the
    oracle's J v and J^T w (and so nc_jvp / nc_jtvp)."""
    prob, bc, gp, gam, x = make_pair(nc, c)
    J = prob.jacobian(x, gam)
    xd, gd = dev(x), dev(gam)
    gp.linearize(xd, gd)
    rng = np.random.default_rng(c["seed"] + 17)
    for s in range(3):
        v = rng.standard_normal(prob.g.ndof)
        assert rel(host(gp.jvp_lin(dev(v))), J @ v) <= TOL64
        assert rel(host(gp.jtvp_lin(dev(v))), J.T @ v) <= TOL64


# grids at least a warp of elements wide, ragged in x and y, a single element
# layer, and the flux patch
WIDE_CASES = [
    dict(nx=32, ny=4, nz=2, Gr=1e4, patch="dirichlet", seed=11),
    dict(nx=40, ny=5, nz=3, Gr=1e5, patch="flux", seed=12),
    dict(nx=37, ny=9, nz=1, Gr=1e3, patch="dirichlet", seed=13),
    dict(nx=64, ny=6, nz=2, Gr=1e4, patch="flux", seed=14),
]


# wider grids: an x-row of exactly one warp, x-rows that end inside a warp (a
# warp spanning two rows), ragged in y and z
WARP_ROW_CASES = [
    dict(nx=32, ny=8, nz=4, Gr=1e4, patch="dirichlet", seed=21),
    dict(nx=40, ny=9, nz=35, Gr=1e5, patch="flux", seed=22),
    dict(nx=67, ny=13, nz=6, Gr=1e3, patch="dirichlet", seed=23),
]


@pytest.mark.parametrize("c", CASES + WIDE_CASES + WARP_ROW_CASES)
def test_fp32_operators(nc, c):
    prob, bc, gp, gam, x = make_pair(nc, c)
    J = prob.jacobian(x, gam)
    f = torch.float32
    xd, gd = dev(x, f), dev(gam, f)
    v = np.random.default_rng(3).standard_normal(prob.g.ndof)
    assert rel(host(gp.residual(xd, gd), (5, -1)), prob.residual(x, gam)) <= TOL32
    vd = dev(v, f)
    jv, jtv = gp.jvp(xd, gd, vd), gp.jtvp(xd, gd, vd)
    assert rel(host(jv), J @ v) <= TOL32
    assert rel(host(jtv), J.T @ v) <= TOL32
    # deterministic: fixed summation order, no atomics
    assert torch.equal(gp.jvp(xd, gd, vd), jv) and torch.equal(gp.jtvp(xd, gd, vd), jtv)
    assert rel(host(gp.diag(xd, gd)), J.diagonal()) <= TOL32


def test_fp32_products_sampled_lines(nc):
    """FP32 J v and J^T w at 100 x 40 x 30 (warps straddle x-rows, 120,000
    elements): whole x-rows (every lane position meets a warp boundary somewhere)
    and z-lines against element-by-element oracle rows, plus random nodes; and
    bitwise repeatable."""
    nx, ny, nz = 100, 40, 30
    prob, bc = oracle_problem(nx, ny, nz, 1.0 / nz, 1e5, 0.71, patch_mode="flux")
    g = prob.g
    rng = np.random.default_rng(41)
    gam = rng.uniform(0.0, 1.0, g.E)
    x = random_bc_state(prob, 42)
    v = rng.standard_normal((5, g.Nn))
    vm = np.where(prob.dmask, 0.0, v)
    lines = [g.node(i, j, k) for (i, j) in [(32, 16), (64, 4), (10, 10), (0, 0), (100, 40),
                                            (99, 7)] for k in range(nz + 1)]
    rows = [g.node(i, j, k) for (j, k) in [(4, 15), (17, 29), (0, 30), (40, 0), (23, 1)]
            for i in range(nx + 1)]
    nodes = np.unique(np.array(lines + rows + list(rng.choice(g.Nn, size=40, replace=False))))
    gp = nc.Problem(nc.make_params(nx, ny, nz, 1.0 / nz, 1e5, 0.71, **synth.MATERIAL),
                    nc.cavity_bcs(nc.PATCH_FLUX, 1.0))
    f = torch.float32
    X, Gm, V = dev(x, f), dev(gam, f), dev(v, f)
    idx = torch.tensor(nodes, device="cuda")
    for kind, op in (("jvp", gp.jvp), ("jtvp", gp.jtvp)):
        got = op(X, Gm, V)
        assert torch.equal(op(X, Gm, V), got)
        ref = np.where(prob.dmask[:, nodes], v[:, nodes], sampled_rows(g, prob.prm, x, gam, vm,
                                                                        nodes, kind))
        err = rel(host(got.view(5, -1)[:, idx]), ref)
        assert err <= TOL32, (kind, err)


@pytest.mark.parametrize("c", CASES)
def test_sensitivity_and_objective(nc, c):
    prob, bc, gp, gam, x = make_pair(nc, c)
    lam = np.random.default_rng(5).standard_normal((5, prob.g.Nn))
    s_gpu = host(gp.sensitivity(dev(x), dev(gam), dev(lam)))
    s_or = S.sensitivity(prob, x, gam, lam)
    assert rel(s_gpu, s_or) <= TOL64
    phi, g = gp.objective(dev(x))
    phi_o, g_o = S.objective(prob, bc, x)
    assert phi == pytest.approx(phi_o, rel=1e-13, abs=1e-15)
    assert np.array_equal(host(g, g_o.shape) != 0, g_o != 0)
    if np.any(g_o):  # an empty patch (no face inside it) has a zero gradient
        assert rel(host(g, g_o.shape), g_o) <= 1e-15


def quarter_pair(nc, n=8, Gr=1e3):
    """The paper's quarter cavity (symmetry planes, closed walls, pinned
    pressure, heat-source block) at nx = ny = n, nz = 2n."""
    nx, ny, nz, h = n, n, 2 * n, 1.0 / (2 * n)
    cfg = dict(synth.WORKLOADS["quarter80x80x160_gr1e3"], nx=nx, ny=ny, nz=nz, h=h, Gr=Gr)
    pin = (nx + 1) * (ny + 1) * nz
    bc = G.BCs(vel_bc=(G.NOSLIP, G.SYMMETRY, G.NOSLIP, G.SYMMETRY, G.NOSLIP, G.NOSLIP),
               T_bc=(G.DIRICHLET, G.ADIABATIC, G.DIRICHLET, G.ADIABATIC, G.ADIABATIC, G.DIRICHLET),
               patch_mode=G.PATCH_NONE, p_pin=pin)
    se = synth.source(cfg)
    prob, _ = oracle_problem(nx, ny, nz, h, Gr, cfg["Pr"], bc=bc, se=se, **synth.material(cfg))
    gp = nc.Problem(nc.make_params(nx, ny, nz, h, Gr, cfg["Pr"], **synth.material(cfg)),
                    nc.quarter_bcs(nx, ny, nz))
    gp.set_source(dev(se))
    gam = synth.quarter_design(nx, ny, nz, h, 3)
    return prob, bc, gp, gam


def test_quarter_cavity_operators(nc):
    prob, bc, gp, gam = quarter_pair(nc)
    assert prob.se.sum() > 0 and (gam == 0).sum() >= 1
    fl = gp.bc_flags()
    for f in range(5):
        assert np.array_equal(((fl >> f) & 1).astype(bool), prob.dmask[f])
    x = random_bc_state(prob, 31)
    xd, gd = dev(x), dev(gam)
    assert rel(host(gp.residual(xd, gd), (5, -1)), prob.residual(x, gam)) <= TOL64
    J = prob.jacobian(x, gam)
    v = np.random.default_rng(32).standard_normal(prob.g.ndof)
    assert rel(host(gp.jvp(xd, gd, dev(v))), J @ v) <= TOL64
    assert rel(host(gp.jtvp(xd, gd, dev(v))), J.T @ v) <= TOL64
    phi, g = gp.objective(xd)
    phi_o, g_o = S.objective(prob, bc, x)
    assert phi == pytest.approx(phi_o, rel=1e-13)
    assert rel(host(g, g_o.shape), g_o) <= 1e-14
    lam = np.random.default_rng(33).standard_normal((5, prob.g.Nn))
    assert rel(host(gp.sensitivity(xd, gd, dev(lam))), S.sensitivity(prob, x, gam, lam)) <= TOL64


def test_quarter_cavity_newton_matches_oracle(nc):
    """Quarter cavity with the source block: Newton (FP64 and mixed) against the
    oracle's direct-solve Newton, the whole state (all five fields at every
    node, the solid block's pressure included) to 1e-8 relative, and the thermal
    compliance to 1e-10.  The pressure is the least damped field of the residual
    (a residual reduction of 1e-10 leaves about 1e-7 in p, 1e-9 in u and T), so
    both solves go to 1e-12; the oracle's own direct solves with three column
    orderings and a dense solve agree to 1e-15 there, so the pressure is fully
    determined by the discrete equations."""
    prob, bc, gp, gam = quarter_pair(nc)
    xo, _ = S.newton(prob, gam, np.zeros((5, prob.g.Nn)), rtol=1e-13)
    fo, _ = S.objective(prob, bc, xo)
    for mixed in (0, 1):
        x = torch.zeros(gp.ndof, dtype=torch.float64, device="cuda")
        _, info = gp.newton_solve(dev(gam), x, nc.default_opts(mixed=mixed, rtol_newton=1e-12))
        xh = host(x, (5, -1))
        err = rel(xh, xo)
        assert err <= 1e-8, (mixed, err, info)
        f, _ = gp.objective(x)
        assert f == pytest.approx(fo, rel=1e-10)


def test_adjoint_dot_product_32cube(nc):
    """w^T (J v) = (J^T w)^T v at a size beyond the oracle's (32^3, FP64)."""
    n = 32
    p = nc.make_params(n, n, n, 1.0 / n, 1e5, 0.71, **synth.MATERIAL)
    gp = nc.Problem(p, nc.cavity_bcs())
    rng = np.random.default_rng(11)
    gam = dev(synth.smoothed_random(n, n, n, 1.0 / n, 4))
    x = dev(synth.random_state(n, n, n, 12, (0.5, 0.5, 0.5, 50, 1)))
    gp.impose_dirichlet(x)
    v, w = dev(rng.standard_normal(gp.ndof)), dev(rng.standard_normal(gp.ndof))
    a = torch.dot(w, gp.jvp(x, gam, v)).item()
    b = torch.dot(gp.jtvp(x, gam, w), v).item()
    assert a == pytest.approx(b, rel=1e-12)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_fins64_sampled_rows(nc, prec):
    """64^3 fins workload in the launch configuration the benchmark times: J v
    and J^T w rows at 48 sampled nodes against element-by-element oracle rows."""
    name = "fins64_gr1e4"
    cfg = synth.WORKLOADS[name]
    gp = nc.Problem.from_workload(name)
    n = cfg["nx"]
    prob, bc = oracle_problem(n, n, n, cfg["h"], cfg["Gr"], cfg["Pr"])
    gam = synth.design(name)
    x = random_bc_state(prob, 21)
    rng = np.random.default_rng(22)
    v = rng.standard_normal((5, prob.g.Nn))
    dt = torch.float64 if prec == "f64" else torch.float32
    tol = TOL64 if prec == "f64" else TOL32
    Jv = host(gp.jvp(dev(x, dt), dev(gam, dt), dev(v, dt)), (5, -1))
    JTw = host(gp.jtvp(dev(x, dt), dev(gam, dt), dev(v, dt)), (5, -1))
    nodes = rng.choice(prob.g.Nn, size=48, replace=False)
    vm = np.where(prob.dmask, 0.0, v)
    got_all = [("jvp", Jv), ("jtvp", JTw)]
    if prec == "f64":  # the benchmark's FP64 step: linearisation store, then the products
        X, Gm = dev(x), dev(gam)
        gp.linearize(X, Gm)
        got_all += [("jvp", host(gp.jvp_lin(dev(v)), (5, -1))),
                    ("jtvp", host(gp.jtvp_lin(dev(v)), (5, -1)))]
    for kind, got in got_all:
        ref = sampled_rows(prob.g, prob.prm, x, gam, vm, nodes, kind)
        ref = np.where(prob.dmask[:, nodes], v[:, nodes], ref)
        err = rel(got[:, nodes], ref)
        assert err <= tol, (kind, err)


def test_largest_config_sampled_rows(nc):
    """192 x 192 x 384 (71.7M unknowns, the largest workload): J v and J^T w in FP32
    (the operator of the mixed solves) and from the FP64 linearisation store (the
    FP64 path) at 40 sampled nodes -- the corners, patch and top-face nodes and
    random interior ones -- against element-by-element oracle rows."""
    from oracle import element as El
    from oracle import grid as G
    from tests.helpers import oracle_bcs
    name = "tall192x192x384_gr1e6"
    cfg = synth.WORKLOADS[name]
    g = G.Grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["h"])
    m, dv = G.dirichlet(g, oracle_bcs(cfg["patch"]))
    x = np.where(m, dv, synth.random_state(g.nx, g.ny, g.nz, 31, (0.5, 0.5, 0.5, 50, 1)))
    gam = synth.design(name)
    prm = El.Params(cfg["h"], cfg["Gr"], cfg["Pr"], **synth.MATERIAL)
    rng = np.random.default_rng(32)
    v = rng.standard_normal((5, g.Nn))
    vm = np.where(m, 0.0, v)
    nx1, ny1 = g.nx + 1, g.ny + 1
    special = [0, g.nx, g.Nn - 1, g.Nn - nx1, g.node(96, 96, 0), g.node(64, 64, 0),
               g.node(128, 128, 0), g.node(100, 90, 384), g.node(0, 96, 200), g.node(192, 5, 7)]
    nodes = np.array(special + list(rng.choice(g.Nn, size=30, replace=False)))
    gp = nc.Problem.from_workload(name)
    refs = {k: np.where(m[:, nodes], v[:, nodes], sampled_rows(g, prm, x, gam, vm, nodes, k))
            for k in ("jvp", "jtvp")}
    X32, G32, V32 = dev(x, torch.float32), dev(gam, torch.float32), dev(v, torch.float32)
    idx = torch.tensor(nodes, device="cuda")
    pick = lambda t: host(t.view(5, -1)[:, idx])
    assert rel(pick(gp.jvp(X32, G32, V32)), refs["jvp"]) <= TOL32
    assert rel(pick(gp.jtvp(X32, G32, V32)), refs["jtvp"]) <= TOL32
    del X32, G32, V32
    X, Gm, V = dev(x), dev(gam), dev(v)
    gp.linearize(X, Gm)
    err = rel(pick(gp.jvp_lin(V)), refs["jvp"])
    assert err <= TOL64, ("jvp_lin", err)
    err = rel(pick(gp.jtvp_lin(V)), refs["jtvp"])
    assert err <= TOL64, ("jtvp_lin", err)


def test_largest_config_mixed_solve_matches_fp64(nc):
    """192 x 192 x 384 (71.7M unknowns, Gr = 1e6, flux-heated patch): the
    mixed-precision state, adjoint and sensitivity solve of one design iteration
    agrees with the plain FP64 solve on the same GPU to 1e-8 (state and the
    sensitivities of all 14.16M elements), as the benchmark's design iteration
    runs it: a cold mixed state solve of the design by grid sequencing, one
    synthetic design step, then per precision the warm Newton solve to 1e-8, the
    objective's gradient, the adjoint to 1e-10 and the sensitivities.  The oracle's
    direct solves do not reach this size; their agreement with both modes is
    tested at 12^3 and 8^3."""
    name = "tall192x192x384_gr1e6"
    prob = nc.Problem.from_workload(name, patch="flux")
    g0h = synth.design(name)
    g0 = dev(g0h)
    g1 = dev(synth.design_step(name, g0h, 77))
    x0 = torch.zeros(prob.ndof, dtype=torch.float64, device="cuda")
    prob.newton_solve_sequenced(g0, x0, nc.default_opts(mixed=1, ramp_steps=3))
    out = {}
    for mixed in (1, 0):
        x = x0.clone()
        _, info = prob.newton_solve(g1, x, nc.default_opts(mixed=mixed, rtol_newton=1e-8,
                                                           ramp_steps=3))
        assert info["status"] == "NC_OK", (mixed, info["status"])
        _, dphi = prob.objective(x)
        lam, ainfo = prob.adjoint_solve(x, g1, -dphi, opts=nc.default_opts(mixed=mixed))
        assert ainfo["status"] == "NC_OK", (mixed, ainfo["status"])
        out[mixed] = (x, prob.sensitivity(x, g1, lam))
        del lam, dphi
    (xm, sm), (xd, sd) = out[1], out[0]
    err_x = float(torch.linalg.norm(xm - xd) / torch.linalg.norm(xd))
    err_s = float(torch.linalg.norm(sm - sd) / torch.linalg.norm(sd))
    assert err_x <= 1e-8 and err_s <= 1e-8, (err_x, err_s)


def test_newton_matches_oracle_cfg0(nc):
    """cavity12_gr1e3: Newton-FGMRES-multigrid (FP64 and mixed) converges to the
    oracle's direct-solve Newton solution."""
    name = "cavity12_gr1e3"
    cfg = synth.WORKLOADS[name]
    prob, bc = oracle_problem(12, 12, 12, cfg["h"], cfg["Gr"], cfg["Pr"])
    gam = synth.design(name)
    xo, _ = S.newton(prob, gam, np.zeros((5, prob.g.Nn)), rtol=1e-12)
    gp = nc.Problem.from_workload(name)
    for mixed in (0, 1):
        x = torch.zeros(gp.ndof, dtype=torch.float64, device="cuda")
        _, info = gp.newton_solve(dev(gam), x, nc.default_opts(mixed=mixed, rtol_newton=1e-10))
        assert info["status"] == "NC_OK"
        assert rel(host(x), xo.ravel()) <= 1e-8, info


def test_adjoint_and_sensitivity_match_oracle(nc):
    """Flux-patch cavity at 8^3: adjoint solve and sensitivities against the
    oracle's direct adjoint (the adjoint at the oracle's converged state).  The
    refinement stops on ||rhs - J^T lambda|| <= rtol_adjoint ||rhs||, which bounds
    the solution error by cond(J) rtol_adjoint: at the default 1e-10 the residual
    is checked and the adjoint and the sensitivities are compared with the
    oracle's to 1e-8; a solve to 1e-11 is compared to 1e-9."""
    n, Gr = 8, 1e4
    prob, bc = oracle_problem(n, n, n, 1.0 / n, Gr, 0.71, patch_mode="flux")
    gam = synth.smoothed_random(n, n, n, 1.0 / n, 3)
    xo, _ = S.newton(prob, gam, np.zeros((5, prob.g.Nn)), rtol=1e-13)
    phi, dphi = S.objective(prob, bc, xo)
    lam_o = S.adjoint(prob, xo, gam, -dphi)
    sens_o = S.sensitivity(prob, xo, gam, lam_o)
    p = nc.make_params(n, n, n, 1.0 / n, Gr, 0.71, **synth.MATERIAL)
    gp = nc.Problem(p, nc.cavity_bcs(nc.PATCH_FLUX, 1.0))
    for mixed in (0, 1):
        lam, info = gp.adjoint_solve(dev(xo), dev(gam), dev(-dphi),
                                     opts=nc.default_opts(mixed=mixed))
        assert info["res_final"] <= 1e-10 * info["res0"], info
        assert rel(host(lam), lam_o.ravel()) <= 1e-8, info
        sens = host(gp.sensitivity(dev(xo), dev(gam), lam))
        assert rel(sens, sens_o) <= 1e-8
        lam, info = gp.adjoint_solve(dev(xo), dev(gam), dev(-dphi),
                                     opts=nc.default_opts(mixed=mixed, rtol_adjoint=1e-11))
        assert rel(host(lam), lam_o.ravel()) <= 1e-9, info
        sens = host(gp.sensitivity(dev(xo), dev(gam), lam))
        assert rel(sens, sens_o) <= 1e-9


def test_errors_are_status_codes(nc):
    p = nc.make_params(4, 4, 4, 0.25, 1e3, 0.71)
    gp = nc.Problem(p, nc.cavity_bcs())
    x = torch.zeros(gp.ndof, dtype=torch.float64, device="cuda")
    gam = torch.full((gp.E,), float("nan"), dtype=torch.float64, device="cuda")
    _, info = gp.newton_solve(gam, x, check=False)
    assert info["status"] == "NC_ERR_NAN"
    # bad sizes -> NC_ERR_ARG without touching the device
    bad = nc.make_params(0, 4, 4, 0.25, 1e3, 0.71)
    ctx = nc._ctx()
    import ctypes
    assert nc.lib.nc_setup(ctypes.byref(bad), ctypes.byref(nc.cavity_bcs()), ctypes.byref(ctx)) == 1
    assert nc.lib.nc_residual(gp.ctx, None, None, None, 0, None) == 1


@pytest.mark.parametrize("n,k,ldv", [(1001, 1, 1024), (1001, 5, 1003), (5 * 33 ** 3, 8, 5 * 33 ** 3 + 3),
                                     (5 * 33 ** 3, 30, 179712), (6, 3, 6)])
def test_arnoldi_orth_matches_oracle(nc, n, k, ldv):
    """FGMRES orthogonalisation step (classical Gram-Schmidt twice, Sec. 5.2)
    through nc_arnoldi_orth against the oracle's plain two-pass Gram-Schmidt:
    FP64 to 1e-12, FP32 to 1e-5 (inputs rounded to FP32, sums of n/155k terms
    per thread in FP32).  Aligned (ldv a multiple of 4) and unaligned column
    strides, a ragged length, k from 1 to 30, two calls in a row."""
    rng = np.random.default_rng(n + k)
    Vh = np.linalg.qr(rng.standard_normal((n, k)))[0].T
    gp = nc.Problem(nc.make_params(2, 2, 2, 0.5, 1e3, 0.71), nc.cavity_bcs())
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        Vd = torch.zeros(k * ldv, dtype=dt, device="cuda")
        for i in range(k):
            Vd[i * ldv:i * ldv + n] = torch.tensor(Vh[i], dtype=dt)
        Vr = np.stack([host(Vd[i * ldv:i * ldv + n]) for i in range(k)])
        for rep in range(2):
            w0 = Vh.T @ rng.standard_normal(k) + rng.standard_normal(n)
            w = dev(w0, dt)
            w0r = host(w)
            h = gp.arnoldi_orth(Vd, w, k, ldv)
            ho, nuo, qo = S.gram_schmidt_twice(Vr, w0r)
            assert rel(h[:k], ho) <= tol and abs(h[k] - nuo) <= tol * nuo, (dt, rep)
            assert rel(host(w), qo) <= tol, (dt, rep)


def _mma_case(rng, n):
    x = rng.uniform(0.05, 0.95, n)
    xo1 = np.clip(x + rng.normal(0, 0.05, n), 0, 1)
    xo2 = np.clip(xo1 + rng.normal(0, 0.05, n), 0, 1)
    low, upp = x - rng.uniform(0.05, 0.6, n), x + rng.uniform(0.05, 0.6, n)
    df0 = rng.normal(0, 1, n) * rng.uniform(0, 3, n)
    df1 = -rng.uniform(0.5, 1.5, n) / n
    return x, xo1, xo2, low, upp, df0, df1


@pytest.mark.parametrize("n,k,f1", [(10007, 0, 0.03), (10007, 1, 0.03), (10007, 4, 0.03),
                                    (10007, 4, -0.5), (257, 7, 0.01)])
def test_mma_update_matches_oracle(nc, n, k, f1):
    """One MMA iteration (Sec. 3.2, Svanberg 1987) through nc_mma_update against
    the oracle's step on the active variables (a seeded mask of about 60 %):
    new iterate, asymptotes and multiplier to 1e-10; inactive variables keep
    their value; the history shifts; the reported change is max |x_new - x|.
    Cases: the first two iterations (fixed asymptotes), later iterations
    (adapted asymptotes), an inactive constraint (multiplier 0) and a small
    ragged size.  The objective gradient goes in divided by 4 with
    df0_scale = 4."""
    from oracle import mma as M
    rng = np.random.default_rng(n + k)
    x, xo1, xo2, low, upp, df0, df1 = _mma_case(rng, n)
    a = rng.uniform(0, 1, n) < 0.6
    yo, Lo, Uo, lo = M.mma_step(k, x[a], xo1[a], xo2[a], low[a], upp[a], f1, df0[a], df1[a],
                                move=0.2)
    gp = nc.Problem(nc.make_params(2, 2, 2, 0.5, 1e3, 0.71), nc.cavity_bcs())
    X, X1, X2, L, U = dev(x), dev(xo1), dev(xo2), dev(low), dev(upp)
    lam, chg = gp.mma_update(k, X, X1, X2, L, U, dev(df0 / 4.0), f1, dev(df1),
                             active=torch.tensor(a.astype(np.uint8), device="cuda"),
                             df0_scale=4.0)
    assert lam == pytest.approx(lo, rel=1e-10, abs=1e-300)
    assert np.max(np.abs(host(X)[a] - yo)) <= 1e-10
    assert np.array_equal(host(X)[~a], x[~a])
    assert np.array_equal(host(X1), x) and np.array_equal(host(X2), xo1)
    assert np.max(np.abs(host(L)[a] - Lo)) <= 1e-12 and np.max(np.abs(host(U)[a] - Uo)) <= 1e-12
    assert chg == pytest.approx(np.max(np.abs(host(X) - x)), rel=1e-12)


def test_volume_matches_oracle(nc):
    """Normalised volume constraint (Sec. 3.2) and its gradient through nc_volume
    against the oracle's (oracle.mma.volume_constraint), with and without a
    design mask, on a ragged size; a design at exactly the volume fraction gives 0."""
    from oracle import mma as M
    rng = np.random.default_rng(21)
    n = 33333
    g = rng.uniform(0, 1, n)
    act = rng.uniform(0, 1, n) < 0.3
    gp = nc.Problem(nc.make_params(2, 2, 2, 0.5, 1e3, 0.71), nc.cavity_bcs())
    grad = torch.empty(n, dtype=torch.float64, device="cuda")
    am = torch.tensor(act.astype(np.uint8), device="cuda")
    v = gp.volume(dev(g), am, vf=0.05, grad=grad)
    vo, go = M.volume_constraint(g, act, 0.05)
    assert v == pytest.approx(vo, rel=1e-13)
    assert np.allclose(host(grad), go, rtol=1e-15, atol=0)
    assert gp.volume(dev(g), None, vf=0.5) == pytest.approx(M.volume_constraint(g, None, 0.5)[0],
                                                           rel=1e-13)
    at_vf = np.where(act, 0.95, g)
    assert abs(gp.volume(dev(at_vf), am, vf=0.05)) <= 1e-13


def test_design_map(nc):
    """Physical design from filtered variables: clamp on the design variables,
    fixed values elsewhere; a gradient restricted to the design variables."""
    rng = np.random.default_rng(22)
    n = 1001
    v = rng.normal(0.5, 0.6, n)
    act = rng.uniform(0, 1, n) < 0.5
    fixed = rng.uniform(0, 1, n)
    gp = nc.Problem(nc.make_params(2, 2, 2, 0.5, 1e3, 0.71), nc.cavity_bcs())
    a = torch.tensor(act.astype(np.uint8), device="cuda")
    out = gp.design_map(dev(v), a, dev(fixed), 0.0, 1.0)
    assert np.array_equal(host(out), np.where(act, np.clip(v, 0, 1), fixed))
    out = gp.design_map(dev(v), a)
    assert np.array_equal(host(out), np.where(act, v, 0.0))
