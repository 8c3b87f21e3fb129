"""GPU parity of the multigrid level operators (Sec. 5.2) through nc_mg_apply:
Galerkin coarse operators P^T A P (two levels deep) and rediscretised coarse
operators against the FP64 oracle, and Newton with Galerkin coarse operators
against the oracle's direct-solve solution.

Tolerances as in test_gpu_parity: FP64 relative L2 <= 1e-12 on random
BC-consistent states; FP32 <= 2e-4."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import multigrid as MG  # noqa: E402
from oracle import solve as S  # noqa: E402
from paper_1508_04596_gb300 import synth  # noqa: E402
from tests.helpers import oracle_problem, random_bc_state  # noqa: E402


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


def host(t):
    return t.detach().double().cpu().numpy()


def hierarchy(n, Gr, seed, levels):
    """Oracle problems of the first `levels` levels of an n^3 flux-patch cavity."""
    probs = []
    for l in range(levels):
        m = n >> l
        probs.append(oracle_problem(m, m, m, 1.0 / m, Gr, 0.71, patch_mode="flux")[0])
    p0 = probs[0]
    x = random_bc_state(p0, seed)
    gam = synth.smoothed_random(n, n, n, 1.0 / n, seed)
    return probs, x, gam


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-4)])
def test_galerkin_levels_match_oracle(nc, prec, tol):
    """8^3 cavity (levels 8^3, 4^3, 2^3): the Galerkin operators of levels 1 and 2,
    and their transposes, applied to random vectors, against P^T J P and
    P^T (P^T J P) P assembled by the oracle from its complex-step Jacobian."""
    probs, x, gam = hierarchy(8, 1e4, 3, 3)
    J = probs[0].jacobian(x, gam)
    A = [J]
    for l in (1, 2):
        P = MG.prolongation(probs[l - 1].g, probs[l].g, probs[l - 1].dmask, probs[l].dmask)
        A.append(MG.galerkin(A[l - 1], P, probs[l].dmask))
    p = nc.make_params(8, 8, 8, 1.0 / 8, 1e4, 0.71, **synth.MATERIAL)
    gp = nc.Problem(p, nc.cavity_bcs(nc.PATCH_FLUX, 1.0))
    dt = torch.float64 if prec == "f64" else torch.float32
    rng = np.random.default_rng(5)
    for l in (1, 2):
        assert gp.level_dims(l) == (8 >> l,) * 3
        v = rng.standard_normal(A[l].shape[0])
        vr = host(dev(v, dt))
        for tr in (False, True):
            out = gp.mg_apply(l, dev(x), dev(gam), dev(v, dt), transpose=tr, galerkin=True)
            ref = (A[l].T if tr else A[l]) @ vr
            assert rel(host(out), ref) <= tol, (l, tr)


def test_rediscretised_level_matches_oracle(nc):
    """Level 1 of the rediscretised hierarchy: the Jacobian of the coarse grid at
    the injected state (the fine values at the even nodes) and the mean design of
    the eight children, against the oracle's coarse Jacobian at those inputs."""
    probs, x, gam = hierarchy(8, 1e4, 4, 2)
    g0, g1 = probs[0].g, probs[1].g
    ijk = g1.node_ijk()
    xc = x[:, g0.node(2 * ijk[:, 0], 2 * ijk[:, 1], 2 * ijk[:, 2])]
    gc = gam.reshape(8, 8, 8).reshape(4, 2, 4, 2, 4, 2).mean(axis=(1, 3, 5)).ravel()
    Jc = probs[1].jacobian(xc, gc)
    p = nc.make_params(8, 8, 8, 1.0 / 8, 1e4, 0.71, **synth.MATERIAL)
    gp = nc.Problem(p, nc.cavity_bcs(nc.PATCH_FLUX, 1.0))
    v = np.random.default_rng(6).standard_normal(Jc.shape[0])
    for tr in (False, True):
        out = gp.mg_apply(1, dev(x), dev(gam), dev(v), transpose=tr, galerkin=False)
        assert rel(host(out), (Jc.T if tr else Jc) @ v) <= 1e-12, tr


def test_newton_with_galerkin_coarse_operators(nc):
    """cavity12_gr1e3 (levels 12^3, 6^3, 3^3; the coarsest solved by the dense
    inverse of its Galerkin stencil): Newton-FGMRES-multigrid with Galerkin
    coarse operators, FP64 and mixed, reaches the oracle's direct-solve Newton
    solution to 1e-8, and the adjoint of the 8^3 flux cavity solved to 1e-11
    matches the oracle's direct adjoint to 1e-8."""
    name = "cavity12_gr1e3"
    cfg = synth.WORKLOADS[name]
    prob, _ = oracle_problem(12, 12, 12, cfg["h"], cfg["Gr"], cfg["Pr"])
    gam = synth.design(name)
    xo, _ = S.newton(prob, gam, np.zeros((5, prob.g.Nn)), rtol=1e-12)
    gp = nc.Problem.from_workload(name)
    for mixed in (0, 1):
        x = torch.zeros(gp.ndof, dtype=torch.float64, device="cuda")
        _, info = gp.newton_solve(dev(gam), x, nc.default_opts(mixed=mixed, rtol_newton=1e-10,
                                                                galerkin=1))
        assert info["status"] == "NC_OK", info
        assert rel(host(x), xo.ravel()) <= 1e-8, info
    n = 8
    pa, bc = oracle_problem(n, n, n, 1.0 / n, 1e4, 0.71, patch_mode="flux")
    ga = synth.smoothed_random(n, n, n, 1.0 / n, 3)
    xa, _ = S.newton(pa, ga, np.zeros((5, pa.g.Nn)), rtol=1e-13)
    phi, dphi = S.objective(pa, bc, xa)
    lam_o = S.adjoint(pa, xa, ga, -dphi)
    p = nc.make_params(n, n, n, 1.0 / n, 1e4, 0.71, **synth.MATERIAL)
    gq = nc.Problem(p, nc.cavity_bcs(nc.PATCH_FLUX, 1.0))
    for mixed in (0, 1):
        lam, info = gq.adjoint_solve(dev(xa), dev(ga), dev(-dphi),
                                     opts=nc.default_opts(mixed=mixed, rtol_adjoint=1e-11,
                                                          galerkin=1))
        assert info["status"] == "NC_OK" and rel(host(lam), lam_o.ravel()) <= 1e-8, info
