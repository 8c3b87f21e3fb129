"""GPU parity of the assembled Jacobian (nc_assemble, nc_stencil_apply and the
solvers' `assembled` option) against the FP64 oracle.

The stencil is compared entry by entry with the oracle's complex-step Jacobian:
on small grids the whole matrix, on the 64^3 benchmark grid the rows of sampled
nodes.  Tolerances as for the matrix-free operators: FP64 relative (Frobenius /
L2) <= 1e-12, FP32 products <= 2e-4.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import scipy.sparse as sp  # noqa: E402
from scipy.sparse.linalg import norm as spnorm  # noqa: E402

from oracle import solve as S  # noqa: E402
from paper_1508_04596_gb300 import synth  # noqa: E402
from tests.helpers import (oracle_problem, random_bc_state, sampled_rows,  # noqa: E402
                           sampled_stencil_rows, stencil_to_csr)
from tests.test_gpu_parity import (CASES, TOL32, TOL64, dev, host, make_pair,  # noqa: E402
                                   quarter_pair, rel)


@pytest.fixture(scope="module")
def nc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1508_04596_gb300 import nc as ncmod
    return ncmod


@pytest.mark.parametrize("c", CASES)
def test_assembled_matches_oracle_jacobian(nc, c):
    prob, bc, gp, gam, x = make_pair(nc, c)
    J = sp.csr_matrix(prob.jacobian(x, gam))
    xd, gd = dev(x), dev(gam)
    Sd = gp.assemble(xd, gd)
    A = stencil_to_csr(host(Sd), c["nx"], c["ny"], c["nz"])
    assert spnorm(A - J) <= TOL64 * spnorm(J)
    rng = np.random.default_rng(c["seed"] + 27)
    for _ in range(2):
        v = rng.standard_normal(prob.g.ndof)
        assert rel(host(gp.stencil_apply(Sd, dev(v))), J @ v) <= TOL64
        assert rel(host(gp.stencil_apply(Sd, dev(v), transpose=True)), J.T @ v) <= TOL64
    # deterministic: a second assembly is bitwise identical
    assert torch.equal(gp.assemble(xd, gd), Sd)
    # FP32 assembly and products
    x32, g32 = dev(x, torch.float32), dev(gam, torch.float32)
    S32 = gp.assemble(x32, g32)
    v = rng.standard_normal(prob.g.ndof)
    assert rel(host(gp.stencil_apply(S32, dev(v, torch.float32))), J @ v) <= TOL32
    assert rel(host(gp.stencil_apply(S32, dev(v, torch.float32), transpose=True)), J.T @ v) <= TOL32


def test_assembled_quarter_cavity(nc):
    """The paper's quarter cavity at 8 x 8 x 16 (symmetry planes, pinned pressure,
    heat-source block, the paper's material parameters): the assembled stencil
    equals the oracle's Jacobian, FP64 and FP32."""
    prob, bc, gp, gam = quarter_pair(nc)
    x = random_bc_state(prob, 35)
    J = sp.csr_matrix(prob.jacobian(x, gam))
    A = stencil_to_csr(host(gp.assemble(dev(x), dev(gam))), prob.g.nx, prob.g.ny, prob.g.nz)
    assert spnorm(A - J) <= TOL64 * spnorm(J)
    S32 = gp.assemble(dev(x, torch.float32), dev(gam, torch.float32))
    v = np.random.default_rng(36).standard_normal(prob.g.ndof)
    assert rel(host(gp.stencil_apply(S32, dev(v, torch.float32))), J @ v) <= TOL32


def test_assembled_fins64_sampled_rows(nc):
    """The 64^3 fins workload of the benchmark: stencil rows of 32 sampled nodes
    (corners, patch, top face and random ones) against the oracle's element
    Jacobians, and the assembled product at those rows."""
    name = "fins64_gr1e4"
    cfg = synth.WORKLOADS[name]
    n = cfg["nx"]
    prob, bc = oracle_problem(n, n, n, cfg["h"], cfg["Gr"], cfg["Pr"])
    g = prob.g
    gam = synth.design(name)
    x = random_bc_state(prob, 41)
    rng = np.random.default_rng(42)
    special = [0, n, g.Nn - 1, g.node(n // 2, n // 2, 0), g.node(n // 3, n // 3, 0),
               g.node(20, 40, n), g.node(0, 30, 30), g.node(64, 3, 10)]
    nodes = np.array(special + list(rng.choice(g.Nn, size=24, replace=False)))
    gp = nc.Problem.from_workload(name)
    Sd = gp.assemble(dev(x), dev(gam))
    idx = torch.tensor(nodes, device="cuda")
    got = host(Sd.view(675, -1)[:, idx]).reshape(27, 5, 5, -1).transpose(3, 0, 1, 2)
    ref = sampled_stencil_rows(g, prob.prm, x, gam, prob.dmask, nodes)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= TOL64, ("stencil rows", err)
    v = rng.standard_normal((5, g.Nn))
    vm = np.where(prob.dmask, 0.0, v)
    out = host(gp.stencil_apply(Sd, dev(v)), (5, -1))[:, nodes]
    rows = np.where(prob.dmask[:, nodes], v[:, nodes], sampled_rows(g, prob.prm, x, gam, vm, nodes, "jvp"))
    err = rel(out, rows)
    assert err <= TOL64, ("assembled product rows", err)


def test_newton_with_assembled_operators(nc):
    """cavity12_gr1e3 with every level's operator assembled (FP64 and mixed, with
    and without Galerkin coarse operators): Newton reaches the oracle's direct
    solution."""
    name = "cavity12_gr1e3"
    cfg = synth.WORKLOADS[name]
    prob, bc = oracle_problem(12, 12, 12, cfg["h"], cfg["Gr"], cfg["Pr"])
    gam = synth.design(name)
    xo, _ = S.newton(prob, gam, np.zeros((5, prob.g.Nn)), rtol=1e-12)
    gp = nc.Problem.from_workload(name)
    its = {}
    for mixed, galerkin, assembled in ((0, 0, 0), (0, 0, 1), (1, 0, 1), (0, 1, 1)):
        x = torch.zeros(gp.ndof, dtype=torch.float64, device="cuda")
        _, info = gp.newton_solve(dev(gam), x, nc.default_opts(
            mixed=mixed, galerkin=galerkin, assembled=assembled, rtol_newton=1e-10))
        assert info["status"] == "NC_OK", info
        assert rel(host(x), xo.ravel()) <= 1e-8, info
        its[(mixed, galerkin, assembled)] = info["lin_its_total"]
    # the assembled operator is the matrix-free one up to rounding
    assert abs(its[(0, 0, 1)] - its[(0, 0, 0)]) <= 2, its


def test_adjoint_with_assembled_operators(nc):
    """Flux-patch cavity at 8^3: the adjoint solve on assembled (transposed)
    stencils reaches the oracle's direct adjoint."""
    n, Gr = 8, 1e4
    prob, bc = oracle_problem(n, n, n, 1.0 / n, Gr, 0.71, patch_mode="flux")
    gam = synth.smoothed_random(n, n, n, 1.0 / n, 3)
    xo, _ = S.newton(prob, gam, np.zeros((5, prob.g.Nn)), rtol=1e-13)
    phi, dphi = S.objective(prob, bc, xo)
    lam_o = S.adjoint(prob, xo, gam, -dphi)
    p = nc.make_params(n, n, n, 1.0 / n, Gr, 0.71, **synth.MATERIAL)
    gp = nc.Problem(p, nc.cavity_bcs(nc.PATCH_FLUX, 1.0))
    for mixed in (0, 1):
        lam, info = gp.adjoint_solve(dev(xo), dev(gam), dev(-dphi),
                                     opts=nc.default_opts(mixed=mixed, assembled=1,
                                                          rtol_adjoint=1e-11))
        assert info["status"] == "NC_OK", info
        assert rel(host(lam), lam_o.ravel()) <= 1e-8, info
