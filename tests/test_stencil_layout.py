"""CPU check of the test helpers for the assembled Jacobian: the oracle's
stencil rows (element Jacobians summed per node, in the 27-point block layout
of nc_assemble) equal the oracle's assembled sparse Jacobian, Dirichlet rows and
columns included, on small grids with both patch modes."""
import numpy as np
import pytest
from scipy.sparse.linalg import norm as spnorm

from paper_1508_04596_gb300 import synth
from tests.helpers import oracle_problem, random_bc_state, sampled_stencil_rows, stencil_to_csr


@pytest.mark.parametrize("nx,ny,nz,patch", [(3, 2, 2, "dirichlet"), (2, 3, 4, "flux"), (1, 1, 1, "dirichlet")])
def test_stencil_rows_equal_oracle_jacobian(nx, ny, nz, patch):
    prob, _ = oracle_problem(nx, ny, nz, 1.0 / nx, 1e4, 0.71, patch_mode=patch)
    gam = synth.smoothed_random(nx, ny, nz, 1.0 / nx, 5)
    x = random_bc_state(prob, 6)
    g = prob.g
    rows = sampled_stencil_rows(g, prob.prm, x, gam, prob.dmask, np.arange(g.Nn))
    Sh = rows.transpose(1, 2, 3, 0).ravel()  # [o][f][c][n]
    J = prob.jacobian(x, gam)
    A = stencil_to_csr(Sh, nx, ny, nz)
    assert spnorm(A - J) <= 1e-13 * spnorm(J)
