"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it follows.  None of them re-types the oracle's own
formulas: they check closed forms, exact discrete solutions, printed numbers and
printed derivatives, brute force and finite differences.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import assemble as A
from oracle import element as El
from oracle import grid as G
from oracle import solve as S
from paper_1508_04596_gb300 import synth


def make(nx, ny, nz, h, Gr=1e3, Pr=0.71, bc=None, se=None, force=None, **mat):
    g = G.Grid(nx, ny, nz, h)
    bc = G.BCs() if bc is None else bc
    m, v = G.dirichlet(g, bc)
    kw = dict(synth.MATERIAL)
    kw.update(mat)
    prm = El.Params(h, Gr, Pr, **kw)
    return g, bc, A.Problem(g, prm, m, v, flux=G.neumann_rhs(g, bc), se=se, force=force)


# ---------------------------------------------------------------- counts
def test_dof_counts_printed():
    """Sec. 6.2-6.4: the printed DOF and element counts (tests/golden/paper_dof_counts.txt)
    follow from 5 unknowns on every node of the structured grid."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_dof_counts.txt")
    rows = [l.split()[:5] for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for nx, ny, nz, dof, ne in rows:
        g = G.Grid(int(nx), int(ny), int(nz), 1.0)
        assert g.ndof == int(dof)
        assert g.E == int(ne)


def test_region_counts_12():
    """Benchmark set-up at 12^3: 5x5 patch nodes, 6x6x9 design-column elements."""
    g = G.Grid(12, 12, 12, 1 / 12)
    assert G.patch_nodes(g, G.BCs()).sum() == 25
    assert synth.design_column(12, 12, 12, 1 / 12).sum() == 6 * 6 * 9
    assert G.patch_faces(g, G.BCs()).size == 16


# ---------------------------------------------------------------- interpolation
@pytest.mark.parametrize("q", [0.0, 1.0, 8.0, 881.0])
def test_interpolation_end_points(q):
    """Sec. 2 Eq. (2)-(3) and Sec. 3.1: K(1)=1, K(0)=1/Ck, alpha(1)=0, alpha(0)=alpha_max."""
    prm = El.Params(0.1, 1.0, 1.0, alpha_max=1e5, q_alpha=q, q_f=q, Ck=1e-2)
    assert El.K_of(1.0, prm) == pytest.approx(1.0, rel=1e-15)
    assert El.K_of(0.0, prm) == pytest.approx(100.0, rel=1e-15)
    assert El.alpha_of(1.0, prm) == 0.0
    assert El.alpha_of(0.0, prm) == pytest.approx(1e5, rel=1e-15)


def test_interpolation_monotone_and_convex_factor():
    """Sec. 3.1: larger q pushes intermediate conductivity towards the fluid value
    (penalises intermediate designs), and alpha decreases monotonically to 0."""
    g = np.linspace(0.0, 1.0, 101)
    prev = None
    for q in (0.881, 8.81, 88.1, 881.0):
        prm = El.Params(0.1, 1.0, 1.0, alpha_max=1e5, q_alpha=8.0, q_f=q, Ck=1e-2)
        K = El.K_of(g, prm)
        assert np.all(np.diff(K) < 0)
        if prev is not None:
            assert np.all(K[1:-1] < prev[1:-1])
        prev = K
        assert np.all(np.diff(El.alpha_of(g, prm)) < 0)


# ---------------------------------------------------------------- tau (App. B)
def test_tau_printed_derivative_u():
    """App. B: the printed dtau/du_e equals the (complex-step) derivative of the coded tau.
    Holds only for the reading ||u_e|| = 2-norm of the 24 velocity unknowns."""
    rng = np.random.default_rng(7)
    prm = El.Params(0.05, 1e4, 0.71, alpha_max=1e4)
    for alpha in (0.0 + 1e-9, 30.0, 3e3):
        ue = rng.standard_normal(24) * 5.0
        printed = El.dtau_du_printed(ue, alpha, prm)
        cs = np.empty(24)
        for k in range(24):
            d = np.zeros(24, complex)
            d[k] = 1e-30j
            cs[k] = El.tau_momentum((ue + d) @ (ue + d), alpha, prm).imag / 1e-30
        assert np.allclose(printed, cs, rtol=1e-12, atol=1e-14 * np.abs(cs).max())


def test_tau_printed_derivative_gamma():
    """App. B: the printed dtau/dgamma_e against the complex-step derivative of
    tau(alpha(gamma)).  As printed, the prefactor is tau/tau3; the derivative of
    the printed tau has tau*tau3 there (same form as the printed dtau/du_e, which
    does match), i.e. the printed expression is the derivative times alpha_e^2 =
    tau3^-2.  Reading: the printed prefactor is a typo; the build differentiates
    the printed tau exactly.  This test pins that reading."""
    rng = np.random.default_rng(8)
    prm = El.Params(0.05, 1e4, 0.71, alpha_max=1e4, q_alpha=8.0)
    ue = rng.standard_normal(24) * 3.0
    for gam in (0.1, 0.5, 0.9):
        printed = El.dtau_dgamma_printed(ue, gam, prm)
        t = lambda gm: El.tau_momentum(ue @ ue, El.alpha_of(gm, prm), prm)
        cs = t(gam + 1e-30j).imag / 1e-30
        tau3 = 1.0 / El.alpha_of(gam, prm)
        assert printed * tau3 ** 2 == pytest.approx(cs, rel=1e-12)
        assert abs(printed) > 10 * abs(cs)


def test_tau_limits():
    """App. B: tau is an approximate min of tau1, tau2, tau3."""
    prm = El.Params(0.1, 1.0, 1.0)
    # viscous limit (u = 0, alpha = 0): tau = tau2 = h^2 / (4 Pr)
    assert El.tau_momentum(0.0, 0.0, prm) == pytest.approx(0.1 ** 2 / 4.0, rel=1e-14)
    # Brinkman-dominated: tau -> 1/alpha
    assert El.tau_momentum(0.0, 1e12, prm) == pytest.approx(1e-12, rel=1e-6)
    # convection-dominated: tau -> 4h/||u_e||
    assert El.tau_momentum(1e16, 0.0, prm) == pytest.approx(4 * 0.1 / 1e8, rel=1e-6)


# ---------------------------------------------------------------- Jacobian
def test_jacobian_matches_central_fd():
    """The complex-step J equals central finite differences of R (ragged grid)."""
    g, bc, prob = make(4, 3, 5, 0.2, Gr=1e4)
    rng = np.random.default_rng(3)
    gam = rng.uniform(size=g.E)
    x = prob.impose(rng.standard_normal((5, g.Nn)) * np.array([3, 3, 3, 50, 1.0])[:, None])
    J = prob.jacobian(x, gam)
    for s in range(3):
        v = rng.standard_normal((5, g.Nn))
        v[prob.dmask] = 0.0
        eps = 1e-6
        fd = (prob.residual(x + eps * v, gam) - prob.residual(x - eps * v, gam)) / (2 * eps)
        Jv = (J @ v.ravel()).reshape(5, -1)
        assert np.linalg.norm(fd - Jv) <= 1e-8 * np.linalg.norm(Jv)


def test_dense_brute_force_newton():
    """Brute force on 2^3 and 3^3: the Jacobian built column by column from the
    complex-step derivative of the GLOBAL residual, solved densely, gives the
    same Newton iterates as the assembled sparse J with LU."""
    for n in (2, 3):
        g, bc, prob = make(n, n, n, 1.0 / n, Gr=1e3)
        rng = np.random.default_rng(n)
        gam = rng.uniform(size=g.E)
        x = prob.impose(rng.standard_normal((5, g.Nn)))
        nd = g.ndof
        Jd = np.empty((nd, nd))
        for k in range(nd):
            e = np.zeros(nd)
            e[k] = 1.0
            e = e.reshape(5, -1)
            e[prob.dmask] = 0.0  # Dirichlet columns removed
            col = prob.residual(x + 1j * 1e-30 * e, gam).imag / 1e-30
            col = col.ravel()
            col[prob.dmask.ravel()] = 0.0
            if prob.dmask.ravel()[k]:
                col[k] = 1.0
            Jd[:, k] = col
        Js = prob.jacobian(x, gam).toarray()
        assert np.allclose(Jd, Js, rtol=1e-13, atol=1e-13 * np.abs(Js).max())
        R = prob.residual(x, gam).ravel()
        d_dense = np.linalg.solve(Jd, -R)
        d_sparse = spla.splu(prob.jacobian(x, gam).tocsc()).solve(-R)
        assert np.allclose(d_dense, d_sparse, rtol=1e-10, atol=1e-12 * np.abs(d_dense).max())


def test_quarter_cavity_pressure_is_determined():
    """Sec. 6.1 quarter cavity (symmetry planes, closed walls, pressure pinned at
    one node, a solid heat-source block with s0 = 1e4 and alpha = 1e5): the
    discrete pressure, inside the solid block included, is fixed by the
    equations -- Newton with three different sparse-LU column orderings and with
    a dense solve reaches the same state to round-off in every field."""
    from paper_1508_04596_gb300 import cavity
    n = 6
    nx, ny, nz, h = n, n, 2 * n, 1.0 / (2 * n)
    pin = (nx + 1) * (ny + 1) * nz
    bc = G.BCs(vel_bc=(G.NOSLIP, G.SYMMETRY, G.NOSLIP, G.SYMMETRY, G.NOSLIP, G.NOSLIP),
               T_bc=(G.DIRICHLET, G.ADIABATIC, G.DIRICHLET, G.ADIABATIC, G.ADIABATIC, G.DIRICHLET),
               patch_mode=G.PATCH_NONE, p_pin=pin)
    se = cavity.source(nx, ny, nz, h, True)
    mat = synth.material("quarter80x80x160_gr1e3")
    g, bc, prob = make(nx, ny, nz, h, Gr=1e3, Pr=1.0, bc=bc, se=se, **mat)
    gam = synth.quarter_design(nx, ny, nz, h, 3)
    assert (gam == 0).sum() >= 1 and se.sum() > 0
    sols = []
    for spec in ("COLAMD", "NATURAL", "MMD_AT_PLUS_A", "dense"):
        if spec == "dense":
            ls = lambda J, b: np.linalg.solve(J.toarray(), b)
        else:
            ls = lambda J, b, spec=spec: spla.splu(J.tocsc(), permc_spec=spec).solve(b)
        x, _ = S.newton(prob, gam, np.zeros((5, g.Nn)), rtol=1e-13, linsolve=ls)
        sols.append(x)
    solid = np.zeros(g.Nn, bool)
    solid[prob.conn[gam < 0.5].ravel()] = True
    for x in sols[1:]:
        assert np.linalg.norm(x - sols[0]) <= 1e-12 * np.linalg.norm(sols[0])
        assert np.abs(x[3, solid] - sols[0][3, solid]).max() <= 1e-12 * np.abs(sols[0][3]).max()


# ---------------------------------------------------------------- exact solutions
def hydrostatic_case(Gr, Pr, T0, nx=5, ny=4, nz=6, h=0.2):
    bc = G.BCs(T_bc=(G.DIRICHLET,) * 6, T_val=(T0,) * 6, patch_mode=G.PATCH_DIRICHLET,
               patch_val=T0)
    g, bc, prob = make(nx, ny, nz, h, Gr=Gr, Pr=Pr, bc=bc)
    z = g.node_xyz()[:, 2]
    xs = np.zeros((5, g.Nn))
    xs[3] = Gr * Pr ** 2 * T0 * (z - g.L[2])
    xs[4] = T0
    return g, prob, xs


def test_hydrostatic_rest_is_exact():
    """Sec. 2 Eq. (1): u = 0, uniform T0, p = Gr Pr^2 T0 (z - z_top) solves the
    strong equations (buoyancy balanced by the pressure gradient, p = 0 on the
    traction-free top), is trilinear, so the discrete residual vanishes."""
    g, prob, xs = hydrostatic_case(1e5, 0.71, 1.0)
    gam = np.random.default_rng(0).uniform(size=g.E)
    R = prob.residual(xs, gam)
    scale = 1e5 * 0.71 ** 2 * g.h ** 3
    assert np.abs(R).max() <= 1e-12 * scale


def test_hydrostatic_rest_newton_from_zero():
    g, prob, xs = hydrostatic_case(1e3, 0.71, 2.0)
    gam = np.random.default_rng(1).uniform(size=g.E)
    x, its = S.newton(prob, gam, np.zeros((5, g.Nn)), rtol=1e-13)
    assert np.abs(x - xs).max() <= 1e-9 * np.abs(xs).max()


def q1_laplace_stiffness(h):
    """Textbook exact Q1 cube stiffness  int grad N_a . grad N_b  for edge h:
    h/3 on the diagonal, 0 between edge neighbours, -h/12 between face- and
    body-diagonal corners."""
    Kc = np.empty((8, 8))
    for a in range(8):
        for b in range(8):
            nd = bin(a ^ b).count("1")
            Kc[a, b] = {0: h / 3.0, 1: 0.0, 2: -h / 12.0, 3: -h / 12.0}[nd]
    return Kc


def test_pure_conduction_Gr0_textbook():
    """Gr -> 0 (Sec. 2): no buoyancy, so u = 0, p = 0, and T solves the plain
    heterogeneous conduction problem sum_e K_e K^Q1 T = patch flux, assembled
    here from the textbook Q1 stiffness, independently of the oracle."""
    bc = G.BCs(patch_mode=G.PATCH_FLUX, patch_val=1.0)
    g, bc, prob = make(6, 5, 7, 1 / 6, Gr=0.0, bc=bc)
    gam = synth.smoothed_random(6, 5, 7, 1 / 6, 11)
    gam = np.random.default_rng(2).uniform(size=g.E)
    x, _ = S.newton(prob, gam, np.zeros((5, g.Nn)), rtol=1e-14)
    # independent conduction solve
    conn = g.connectivity()
    Kc = q1_laplace_stiffness(g.h)
    Ke = El.K_of(gam, prob.prm)
    Kg = np.zeros((g.Nn, g.Nn))
    for e in range(g.E):
        Kg[np.ix_(conn[e], conn[e])] += Ke[e] * Kc
    rhs = np.zeros(g.Nn)
    for e in G.patch_faces(g, bc):
        rhs[conn[e, :4]] += 1.0 * g.h ** 2 / 4.0
    dm = prob.dmask[4]
    T = np.zeros(g.Nn)
    free = ~dm
    T[free] = np.linalg.solve(Kg[np.ix_(free, free)], rhs[free])
    assert np.abs(x[0:4]).max() <= 1e-12
    assert np.abs(x[4] - T).max() <= 1e-11 * np.abs(T).max()


def test_slab_dirichlet_linear_profile():
    """1-D slab: T = 1 on the whole bottom, 0 on top, adiabatic sides, Gr = 0 ->
    T = 1 - z / Lz exactly (linear, so exact for Q1)."""
    bc = G.BCs(T_bc=(G.ADIABATIC,) * 4 + (G.ADIABATIC, G.DIRICHLET), patch=(0, 1, 0, 1),
               patch_mode=G.PATCH_DIRICHLET, patch_val=1.0)
    g, bc, prob = make(3, 4, 5, 0.25, Gr=0.0, bc=bc)
    gam = np.random.default_rng(4).uniform(size=g.E)
    x, _ = S.newton(prob, gam, np.zeros((5, g.Nn)), rtol=1e-14)
    z = g.node_xyz()[:, 2]
    # heterogeneous K along z only would bend the profile; use a z-uniform design
    gam2 = np.full(g.E, 0.3)
    x, _ = S.newton(prob, gam2, np.zeros((5, g.Nn)), rtol=1e-14)
    assert np.abs(x[4] - (1.0 - z / g.L[2])).max() <= 1e-12


def test_slab_flux_and_objective():
    """1-D slab heated by flux q on the whole bottom, T = 0 on top, adiabatic
    sides, uniform K: T = q (Lz - z) / K exactly; the mean bottom temperature
    (the objective) is q Lz / K."""
    q = 2.5
    bc = G.BCs(T_bc=(G.ADIABATIC,) * 4 + (G.ADIABATIC, G.DIRICHLET), patch=(0, 1, 0, 1),
               patch_mode=G.PATCH_FLUX, patch_val=q)
    g, bc, prob = make(4, 3, 5, 0.2, Gr=0.0, bc=bc)
    gam = np.full(g.E, 0.4)
    K = El.K_of(0.4, prob.prm)
    x, _ = S.newton(prob, gam, np.zeros((5, g.Nn)), rtol=1e-14)
    z = g.node_xyz()[:, 2]
    assert np.abs(x[4] - q * (g.L[2] - z) / K).max() <= 1e-11 * q * g.L[2] / K
    phi, dphi = S.objective(prob, bc, x)
    assert phi == pytest.approx(q * g.L[2] / K, rel=1e-12)
    assert dphi.sum() == pytest.approx(1.0, rel=1e-14)


def test_thermal_compliance_closed_form():
    """Sec. 3.2: f = int_omega s T dV.  For a uniform temperature T = c it is
    c * sum_e s_e h^3, and its gradient sums to int s dV."""
    bc = G.BCs(patch_mode=G.PATCH_NONE)
    g = G.Grid(4, 3, 5, 0.2)
    se = np.random.default_rng(12).uniform(0.0, 10.0, size=g.E)
    _, bc, prob = make(4, 3, 5, 0.2, bc=bc, se=se)
    x = np.zeros((5, g.Nn))
    x[4] = 1.7
    f, df = S.objective(prob, bc, x)
    assert f == pytest.approx(1.7 * se.sum() * 0.2 ** 3, rel=1e-14)
    assert df.sum() == pytest.approx(se.sum() * 0.2 ** 3, rel=1e-14)


def test_filter_element_matrices_closed_form():
    """Sec. 3.2 filter: the Gauss-integrated Q1 element matrices equal the
    textbook closed forms (stiffness h/3, 0, -h/12, -h/12; mass h^3/216 *
    2^(number of shared coordinates))."""
    from oracle import filter as F
    h = 0.3
    Ke, Me = F.element_matrices(h)
    Kc = q1_laplace_stiffness(h)
    for a in range(8):
        for b in range(8):
            nd = bin(a ^ b).count("1")
            assert Me[a, b] == pytest.approx(h ** 3 / 216.0 * 2 ** (3 - nd), rel=1e-13)
    assert np.allclose(Ke, Kc, rtol=1e-13, atol=1e-15)


def test_filter_preserves_constants_and_volume():
    """Neumann Helmholtz filter: a constant design is unchanged, and the
    design volume sum_e gamma~_e h^3 equals sum_e rho_e h^3 for any rho."""
    from oracle import filter as F
    g = G.Grid(6, 5, 7, 0.1)
    R = 2.5 * g.h
    assert np.allclose(F.apply_filter(g, np.full(g.E, 0.37), R), 0.37, rtol=1e-12)
    rho = np.random.default_rng(13).uniform(size=g.E)
    gt = F.apply_filter(g, rho, R)
    assert gt.sum() == pytest.approx(rho.sum(), rel=1e-12)
    assert gt.std() < rho.std()  # it smooths


def test_filter_cosine_mode_decay():
    """A cosine mode cos(k pi x / L) satisfies the Neumann condition and is an
    eigenfunction of -r^2 lap + 1: it is damped by 1/(1 + r^2 (k pi / L)^2),
    recovered to second order in h."""
    from oracle import filter as F
    errs = []
    for n in (16, 32):
        g = G.Grid(n, 2, 2, 1.0 / n)
        R = 0.1
        r2 = (R / (2 * np.sqrt(3))) ** 2
        c = g.elem_centroids()
        k = 2
        # element averages of the mode (exact cell averages of cos in x)
        x0, x1 = c[:, 0] - g.h / 2, c[:, 0] + g.h / 2
        rho = (np.sin(k * np.pi * x1) - np.sin(k * np.pi * x0)) / (k * np.pi * g.h)
        gt = F.apply_filter(g, rho, R)
        expect = rho / (1.0 + r2 * (k * np.pi) ** 2)
        errs.append(np.abs(gt - expect).max())
    assert errs[1] < errs[0] / 3.0, errs
    assert errs[1] < 1e-2


def test_line_search_closed_form():
    """Sec. 5.1: the step minimises the quadratic through the three norms."""
    for lam_true, c2 in ((0.3, 2.0), (0.8, 0.5), (0.02, 4.0)):
        q = lambda l: c2 * (l - lam_true) ** 2 + 0.1
        lam = S.line_search_length(q(0.0), q(0.5), q(1.0))
        assert lam == pytest.approx(max(lam_true, 0.05), rel=1e-12)
    # concave or minimiser beyond 1: best sampled point, longer on a tie
    assert S.line_search_length(1.0, 0.5, 0.2) == 1.0
    assert S.line_search_length(1.0, 2.0, 3.0) == 0.5
    assert S.line_search_length(1.0, 1.5, 1.5) == 1.0


def test_mirror_symmetry():
    """A design symmetric in x gives a mirror-symmetric converged state:
    u(-x) = -u, and v, w, p, T even (cavity BCs are x-symmetric)."""
    nx, ny, nz = 6, 5, 5
    g, bc, prob = make(nx, ny, nz, 1 / 6, Gr=1e4)
    gam = np.random.default_rng(5).uniform(size=(nz, ny, nx))
    gam = 0.5 * (gam + gam[:, :, ::-1])
    x, _ = S.newton(prob, gam.ravel(), np.zeros((5, g.Nn)), rtol=1e-13)
    xr = x.reshape(5, nz + 1, ny + 1, nx + 1)
    m = xr[:, :, :, ::-1]
    sc = np.abs(x).max(axis=1)
    assert np.abs(xr[0] + m[0]).max() <= 1e-10 * sc[0]
    for f in (1, 2, 3, 4):
        assert np.abs(xr[f] - m[f]).max() <= 1e-10 * max(sc[f], 1e-300)
    assert sc[0] > 1e-3  # the flow is not trivially zero


# ---------------------------------------------------------------- manufactured solution
def mms_fields():
    sympy = pytest.importorskip("sympy")
    X, Y, Z = sympy.symbols("x y z")
    pi = sympy.pi
    psi = sympy.sin(pi * X) * sympy.sin(pi * Y) * sympy.sin(pi * Z)
    phi = sympy.cos(pi * X) * sympy.sin(pi * Y) * sympy.sin(pi * Z) / 2
    A = (phi, 0, psi)
    u = [sympy.diff(A[2], Y) - sympy.diff(A[1], Z), sympy.diff(A[0], Z) - sympy.diff(A[2], X),
         sympy.diff(A[1], X) - sympy.diff(A[0], Y)]
    p = sympy.cos(pi * X) * sympy.cos(pi * Y) * Z
    T = sympy.sin(pi * X) * Y ** 2 + Z
    return sympy, (X, Y, Z), u, p, T


def test_mms_convergence():
    """Sec. 2 Eq. (1): with a smooth divergence-free manufactured solution and
    its body forces, the discrete solution converges at second order in u, T
    (and at least first in p) -- a dropped term, a sign or an index error
    breaks convergence."""
    sympy, (X, Y, Z), u, p, T = mms_fields()
    Gr, Pr, gam0 = 10.0, 1.0, 0.5
    mat = dict(alpha_max=10.0, q_alpha=1.0, q_f=1.0, Ck=0.5)
    prm0 = El.Params(1.0, Gr, Pr, **mat)
    alpha, K = El.alpha_of(gam0, prm0), El.K_of(gam0, prm0)
    xs = (X, Y, Z)
    eg = (0, 0, -1)
    fM = []
    for i in range(3):
        conv = sum(u[j] * sympy.diff(u[i], xs[j]) for j in range(3))
        visc = sum(sympy.diff(sympy.diff(u[i], xs[j]) + sympy.diff(u[j], xs[i]), xs[j])
                   for j in range(3))
        fM.append(conv - Pr * visc + sympy.diff(p, xs[i]) + alpha * u[i]
                  + Gr * Pr ** 2 * eg[i] * T)
    divu = sympy.simplify(sum(sympy.diff(u[j], xs[j]) for j in range(3)))
    assert divu == 0
    fT = sum(u[j] * sympy.diff(T, xs[j]) for j in range(3)) \
        - K * sum(sympy.diff(T, xs[j], 2) for j in range(3))
    fM_l = [sympy.lambdify(xs, f, "numpy") for f in fM]
    fT_l = sympy.lambdify(xs, fT, "numpy")
    ex_l = [sympy.lambdify(xs, f, "numpy") for f in (u + [p, T])]

    def force(xyz):
        a = (xyz[:, 0], xyz[:, 1], xyz[:, 2])
        fm = np.stack([np.broadcast_to(f(*a), xyz[:, 0].shape) for f in fM_l], 1)
        return fm, 0.0, np.broadcast_to(fT_l(*a), xyz[:, 0].shape)

    errs = []
    for n in (4, 8, 12):
        g = G.Grid(n, n, n, 1.0 / n)
        xyz = g.node_xyz()
        exact = np.stack([np.broadcast_to(f(xyz[:, 0], xyz[:, 1], xyz[:, 2]), (g.Nn,))
                          for f in ex_l])
        onb = np.zeros(g.Nn, bool)
        ijk = g.node_ijk()
        for d, nd in enumerate((n, n, n)):
            onb |= (ijk[:, d] == 0) | (ijk[:, d] == nd)
        dm = np.zeros((5, g.Nn), bool)
        dm[[0, 1, 2, 4]] = onb
        dm[3, 0] = True
        prm = El.Params(1.0 / n, Gr, Pr, **mat)
        prob = A.Problem(g, prm, dm, exact.copy(), force=force)
        x, _ = S.newton(prob, np.full(g.E, gam0), np.zeros((5, g.Nn)), rtol=1e-12)
        rms = lambda a: np.sqrt(np.mean(a ** 2))
        errs.append([rms(x[0:3] - exact[0:3]), rms(x[3] - exact[3]), rms(x[4] - exact[4])])
    errs = np.array(errs)
    order = np.log(errs[1] / errs[2]) / np.log(12 / 8)
    assert order[0] > 1.8, (errs, order)   # velocity
    assert order[2] > 1.8, (errs, order)   # temperature
    # pressure (equal-order PSPG, viscous second derivatives dropped from the
    # strong residual): at least first order over 4 -> 12
    assert np.log(errs[0, 1] / errs[2, 1]) / np.log(3.0) > 1.0, errs


# ---------------------------------------------------------------- sensitivities (Sec. 3.2, App. B)
def flux_case(n=4, Gr=1e5):
    bc = G.BCs(patch_mode=G.PATCH_FLUX, patch_val=1.0, patch=(0.25, 0.75, 0.25, 0.75))
    return make(n, n, n, 1.0 / n, Gr=Gr, bc=bc, alpha_max=1e3)


def test_sensitivity_matches_fd_and_consistency_matters():
    """Consistent adjoint sensitivities agree with central FD (step 1e-6) of the
    Newton-converged objective to <= 1e-5 relative; leaving the tau variations
    out of the adjoint (App. B's inconsistent version) is visibly worse."""
    g, bc, prob = flux_case()
    rng = np.random.default_rng(9)
    gam = rng.uniform(0.2, 1.0, size=g.E)
    x = np.zeros((5, g.Nn))
    for Gr in (1e3, 1e4, 1e5):  # convection-dominated, so tau1 matters
        prob.prm.Gr = Gr
        x, _ = S.newton(prob, gam, x, rtol=1e-14, atol=1e-13)
    phi, dphi = S.objective(prob, bc, x)
    lam = S.adjoint(prob, x, gam, -dphi)
    sens = S.sensitivity(prob, x, gam, lam)
    # inconsistent: tau frozen in both the adjoint operator and dR/dgamma
    Jf = prob.jacobian(x, gam, freeze_tau=True)
    lam_f = spla.splu(Jf.T.tocsc()).solve(-dphi.ravel()).reshape(5, -1)
    lam_f[prob.dmask] = 0.0
    dre_f = prob.element_rows(x, gam + 1j * 1e-30, freeze_tau=True).imag / 1e-30
    sens_f = np.einsum("eaf,eaf->e", A.gather(lam_f, prob.conn), dre_f)
    elems = rng.choice(g.E, size=6, replace=False)
    fd = []
    for e in elems:
        vals = []
        for s in (+1, -1):
            gp = gam.copy()
            gp[e] += s * 1e-6
            xp, _ = S.newton(prob, gp, x, rtol=0.0, atol=1e-12, maxit=8)
            vals.append(S.objective(prob, bc, xp)[0])
        fd.append((vals[0] - vals[1]) / 2e-6)
    fd = np.array(fd)
    err = np.abs(sens[elems] - fd).max() / np.abs(fd).max()
    err_f = np.abs(sens_f[elems] - fd).max() / np.abs(fd).max()
    assert err <= 1e-5, err
    assert err_f >= 10 * err, (err, err_f)


def test_adjoint_dot_product():
    """w^T (J v) = (J^T w)^T v for the Dirichlet-modified operator."""
    g, bc, prob = flux_case(3)
    rng = np.random.default_rng(10)
    gam = rng.uniform(size=g.E)
    x = prob.impose(rng.standard_normal((5, g.Nn)))
    J = prob.jacobian(x, gam)
    v, w = rng.standard_normal(g.ndof), rng.standard_normal(g.ndof)
    assert w @ (J @ v) == pytest.approx(v @ (J.T @ w), rel=1e-13)


def test_gram_schmidt_step_against_least_squares():
    """Arnoldi orthogonalisation (Sec. 5.2): for orthonormal V the step returns
    h = V w, nu = the distance from w to span(V) (a least-squares residual from
    numpy's lstsq) and a unit q orthogonal to V with w = V^T h + nu q; a
    nearly dependent w (1e-6 off the span) keeps q orthogonal to V."""
    rng = np.random.default_rng(11)
    n, k = 257, 7
    V = np.linalg.qr(rng.standard_normal((n, k)))[0].T
    for off in (1.0, 1e-6):
        w = V.T @ rng.standard_normal(k) + off * rng.standard_normal(n)
        h, nu, q = S.gram_schmidt_twice(V, w)
        coef, res, _, _ = np.linalg.lstsq(V.T, w, rcond=None)
        assert np.allclose(h, coef, rtol=0, atol=1e-13 * np.linalg.norm(w))
        assert abs(nu - np.sqrt(res[0])) <= 1e-9 * nu
        assert abs(np.linalg.norm(q) - 1.0) <= 1e-14
        assert np.max(np.abs(V @ q)) <= 1e-14
        assert np.linalg.norm(V.T @ h + nu * q - w) <= 1e-13 * np.linalg.norm(w)


def _mma_instance(rng, n):
    x = rng.uniform(0.2, 0.8, n)
    xold1 = np.clip(x + rng.normal(0, 0.05, n), 0, 1)
    xold2 = np.clip(xold1 + rng.normal(0, 0.05, n), 0, 1)
    low, upp = x - 0.3, x + 0.3
    df0 = rng.normal(0, 1, n)
    df1 = -np.ones(n) / n           # a volume-type constraint: sum (1 - x) / n - vf
    f1 = 0.05                       # violated by 0.05, reachable within the move limits
    return x, xold1, xold2, low, upp, f1, df0, df1


def test_volume_constraint_definition():
    """Sec. 3.2 volume constraint: satisfied with equality when the solid volume of
    the design domain is exactly v_f of it, -1 when it is all fluid; elements
    outside the design domain do not count; the gradient equals central
    differences (the constraint is linear); the element size cancels."""
    from oracle import mma as M
    rng = np.random.default_rng(3)
    n, vf = 1000, 0.05
    act = rng.uniform(size=n) < 0.4
    gam = np.where(act, 1.0 - vf, rng.uniform(size=n))
    g, dg = M.volume_constraint(gam, act, vf, h=0.1)
    assert abs(g) <= 1e-12
    assert M.volume_constraint(np.ones(n), act, vf)[0] == pytest.approx(-1.0, abs=1e-15)
    gam2 = gam.copy()
    gam2[~act] = rng.uniform(size=(~act).sum())
    assert M.volume_constraint(gam2, act, vf)[0] == pytest.approx(g, abs=1e-15)
    x = rng.uniform(size=n)
    gx, dgx = M.volume_constraint(x, act, vf, h=0.3)
    for e in (int(np.nonzero(act)[0][3]), int(np.nonzero(~act)[0][5])):
        xp, xm = x.copy(), x.copy()
        xp[e] += 1e-3
        xm[e] -= 1e-3
        fd = (M.volume_constraint(xp, act, vf)[0] - M.volume_constraint(xm, act, vf)[0]) / 2e-3
        assert dgx[e] == pytest.approx(fd, rel=1e-9, abs=1e-13)
    assert M.volume_constraint(x, act, vf, h=2.0)[0] == pytest.approx(gx, rel=1e-13)


def test_mma_subproblem_kkt_and_scipy():
    """MMA (the optimiser of Sec. 3.2): the oracle's step solves its convex
    subproblem.  KKT: each coordinate strictly inside its move limits is
    stationary for the Lagrangian, the constraint is active (its multiplier is
    positive), and on a 6-variable instance the minimiser equals SciPy's SLSQP
    solution of the same subproblem."""
    from scipy.optimize import minimize
    from oracle import mma as M
    rng = np.random.default_rng(3)
    for n, k in ((6, 0), (6, 3), (400, 5)):
        x, xo1, xo2, low, upp, f1, df0, df1 = _mma_instance(rng, n)
        y, L, U, lam = M.mma_step(k, x, xo1, xo2, low, upp, f1, df0, df1, move=0.2)
        al, be = M.bounds(x, L, U, 0.0, 1.0, 0.2)
        p0, q0 = M.approx_coefficients(x, L, U, df0, 1.0)
        p1, q1 = M.approx_coefficients(x, L, U, df1, 1.0)
        assert lam > 0
        assert abs(M.approx_value(f1, x, y, L, U, p1, q1)) <= 1e-12
        grad = (p0 + lam * p1) / (U - y) ** 2 - (q0 + lam * q1) / (y - L) ** 2
        inner = (y > al + 1e-9) & (y < be - 1e-9)
        assert np.all(np.abs(grad[inner]) <= 1e-8 * (1 + np.abs(p0 / (U - y) ** 2)[inner]))
        assert np.all(grad[y <= al + 1e-9] >= -1e-8) and np.all(grad[y >= be - 1e-9] <= 1e-8)
        if n == 6:
            f0t = lambda z: np.sum(p0 / (U - z) + q0 / (z - L))
            con = {"type": "ineq", "fun": lambda z: -M.approx_value(f1, x, z, L, U, p1, q1)}
            r = minimize(f0t, x.copy(), bounds=list(zip(al, be)), constraints=[con],
                         method="SLSQP", options={"ftol": 1e-14, "maxiter": 500})
            assert np.max(np.abs(r.x - y)) <= 1e-6


def test_mma_converges_on_a_convex_problem():
    """MMA iterations on  min sum c_j / x_j  s.t.  sum x_j <= V, 0.01 <= x <= 1,
    whose optimum is x_j = V sqrt(c_j) / sum sqrt(c) (Lagrange conditions; all
    inside the bounds for these c): the objective reaches the optimum to 1e-9
    and the constraint holds."""
    from oracle import mma as M
    rng = np.random.default_rng(4)
    n, V = 50, 20.0
    c = rng.uniform(0.5, 2.0, n)
    xs = V * np.sqrt(c) / np.sum(np.sqrt(c))
    assert np.all((xs > 0.01) & (xs < 1.0))
    x = np.full(n, 0.5)
    xo1 = xo2 = x.copy()
    low, upp = x - 0.5, x + 0.5
    for k in range(80):
        f1 = (np.sum(x) - V) / V
        y, low, upp, lam = M.mma_step(k, x, xo1, xo2, low, upp, f1, -c / x ** 2,
                                      np.ones(n) / V, xmin=0.01, xmax=1.0, move=0.2)
        xo2, xo1, x = xo1, x, y
    assert np.sum(c / x) <= np.sum(c / xs) * (1 + 1e-9)
    assert np.sum(x) <= V * (1 + 1e-12)


def test_mma_approximation_is_first_order_exact():
    """The MMA approximation (Svanberg 1987) agrees with the function and its
    gradient at the expansion point: f~(x) = f(x) and d f~/dy (x) = df/dx for
    gradients of either sign (central differences of f~, step 1e-6)."""
    from oracle import mma as M
    rng = np.random.default_rng(5)
    n = 30
    x = rng.uniform(0.2, 0.8, n)
    low, upp = x - rng.uniform(0.1, 0.5, n), x + rng.uniform(0.1, 0.5, n)
    df = rng.normal(0, 1, n)
    p, q = M.approx_coefficients(x, low, upp, df, 1.0)
    assert M.approx_value(1.7, x, x, low, upp, p, q) == pytest.approx(1.7, abs=1e-15)
    e = 1e-6
    for j in range(n):
        yp, ym = x.copy(), x.copy()
        yp[j] += e
        ym[j] -= e
        fd = (M.approx_value(0.0, x, yp, low, upp, p, q) - M.approx_value(0.0, x, ym, low, upp, p, q)) / (2 * e)
        assert fd == pytest.approx(df[j], rel=1e-6, abs=1e-8)


def test_prolongation_reproduces_trilinear_fields():
    """The multigrid prolongation (Sec. 5.2) is trilinear interpolation: a field
    a + b x + c y + d z + e xyz given at the coarse nodes is reproduced exactly
    at the fine nodes (away from Dirichlet unknowns, none here)."""
    from oracle import multigrid as MG
    gf = G.Grid(4, 6, 2, 0.25)
    gc = MG.coarse_grid(gf)
    none_f, none_c = np.zeros((5, gf.Nn), bool), np.zeros((5, gc.Nn), bool)
    P = MG.prolongation(gf, gc, none_f, none_c)
    f = lambda p: 1.0 + 2 * p[:, 0] - 3 * p[:, 1] + 0.5 * p[:, 2] + 4 * p[:, 0] * p[:, 1] * p[:, 2]
    xc = np.tile(f(gc.node_xyz()), 5)
    assert np.allclose(P @ xc, np.tile(f(gf.node_xyz()), 5), rtol=0, atol=1e-13)


def test_galerkin_conduction_block_is_the_coarse_operator():
    """Variational property of nested Q1 spaces: at rest (u = 0) and uniform
    design, the temperature block of the Jacobian is the conduction stiffness
    K int grad N . grad N (no stabilisation acts at u = 0), and its Galerkin
    projection P^T J_f P equals the coarse grid's own conduction block exactly
    (the trilinear prolongation is the exact embedding of the coarse space)."""
    from oracle import multigrid as MG
    from tests.helpers import oracle_problem
    nf = 4
    pf, _ = oracle_problem(nf, nf, nf, 1.0 / nf, 0.0, 0.71)
    pc, _ = oracle_problem(nf // 2, nf // 2, nf // 2, 2.0 / nf, 0.0, 0.71)
    gam_f, gam_c = np.full(pf.g.E, 0.4), np.full(pc.g.E, 0.4)
    xf, xc = np.zeros((5, pf.g.Nn)), np.zeros((5, pc.g.Nn))
    Jf, Jc = pf.jacobian(xf, gam_f), pc.jacobian(xc, gam_c)
    P = MG.prolongation(pf.g, pc.g, pf.dmask, pc.dmask)
    Ag = MG.galerkin(Jf, P, pc.dmask)
    T = slice(4 * pc.g.Nn, 5 * pc.g.Nn)
    assert abs(Ag[T, T] - Jc[T, T]).max() <= 1e-12 * abs(Jc[T, T]).max()
    # and a wrong prolongation weight (1/4 instead of 1/2) breaks it
    Pb = P.copy()
    Pb.data[np.isclose(Pb.data, 0.5)] = 0.25
    Ab = MG.galerkin(Jf, Pb, pc.dmask)
    assert abs(Ab[T, T] - Jc[T, T]).max() > 1e-3 * abs(Jc[T, T]).max()
