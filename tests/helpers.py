"""Shared test helpers: build oracle problems that mirror a libnc problem, and
compute oracle rows for sampled nodes of large grids."""
import numpy as np

from oracle import assemble as A
from oracle import element as El
from oracle import grid as G
from paper_1508_04596_gb300 import synth


def oracle_bcs(patch_mode="dirichlet", patch_val=1.0):
    mode = G.PATCH_FLUX if patch_mode == "flux" else G.PATCH_DIRICHLET
    return G.BCs(patch_mode=mode, patch_val=patch_val)


def oracle_problem(nx, ny, nz, h, Gr, Pr, patch_mode="dirichlet", se=None, bc=None, **mat):
    g = G.Grid(nx, ny, nz, h)
    bc = oracle_bcs(patch_mode) if bc is None else bc
    m, v = G.dirichlet(g, bc)
    kw = dict(synth.MATERIAL)
    kw.update(mat)
    prm = El.Params(h, Gr, Pr, **kw)
    return A.Problem(g, prm, m, v, flux=G.neumann_rhs(g, bc), se=se), bc


def random_bc_state(prob, seed, scale=(0.5, 0.5, 0.5, 50.0, 1.0)):
    """A random state with the Dirichlet values imposed (||R|| = O(1) scale)."""
    g = prob.g
    x = synth.random_state(g.nx, g.ny, g.nz, seed, scale)
    return prob.impose(x)


def sampled_rows(g, prm, x, gam, v, nodes, kind):
    """Oracle rows (all 5 fields) of J v (kind='jvp'), J^T v ('jtvp') or R ('res',
    without Dirichlet replacement or flux) at the given nodes, computed from the
    complex-step element Jacobians of the up to 8 elements around each node.
    Dirichlet columns must already be zeroed in v by the caller."""
    out = np.zeros((5, len(nodes)))
    nx, ny, nz = g.nx, g.ny, g.nz
    for q, n in enumerate(nodes):
        i = n % (nx + 1)
        j = (n // (nx + 1)) % (ny + 1)
        k = n // ((nx + 1) * (ny + 1))
        for a in range(8):
            ie, je, ke = i - (a & 1), j - ((a >> 1) & 1), k - ((a >> 2) & 1)
            if not (0 <= ie < nx and 0 <= je < ny and 0 <= ke < nz):
                continue
            e = ie + nx * (je + ny * ke)
            conn = [(ie + (b & 1)) + (nx + 1) * ((je + ((b >> 1) & 1)) + (ny + 1) * (ke + ((b >> 2) & 1)))
                    for b in range(8)]
            xe = x[:, conn].T[None]          # [1, 8, 5]
            ve = v[:, conn].T.reshape(40)
            if kind == "res":
                r = El.element_residual(xe, np.array([gam[e]]), prm)[0]
                out[:, q] += r[a]
                continue
            eye = np.eye(40).reshape(40, 8, 5)
            r = El.element_residual(xe + 1e-30j * eye, np.full(40, gam[e]), prm)
            Je = np.transpose(r.imag.reshape(40, 40), (1, 0)) / 1e-30  # Je[row, col]
            if kind == "jvp":
                rows = (Je @ ve).reshape(8, 5)
                out[:, q] += rows[a]
            else:
                # (J^T w)_col: the node is a column of this element's J_e
                cols = (Je.T @ ve).reshape(8, 5)
                out[:, q] += cols[a]
    return out
