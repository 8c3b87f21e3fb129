"""Shared test helpers: build oracle problems that mirror a libnc problem, and
compute oracle rows for sampled nodes of large grids."""
import numpy as np
import scipy.sparse as sparse

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


def sampled_stencil_rows(g, prm, x, gam, dmask, nodes):
    """Oracle rows of J at the given nodes in the 27-point block-stencil layout:
    out[q, o, f, c] = dR(n_q, f) / dx(n_q + offset o, c), o = (dx+1) + 3 (dy+1) +
    9 (dz+1), summed from the complex-step element Jacobians of the elements
    around each node; Dirichlet columns zero, Dirichlet rows identity."""
    out = np.zeros((len(nodes), 27, 5, 5))
    nx, ny, nz = g.nx, g.ny, g.nz
    eye = np.eye(40).reshape(40, 8, 5)
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
            xe = x[:, conn].T[None]
            r = El.element_residual(xe + 1e-30j * eye, np.full(40, gam[e]), prm)
            Je = np.transpose(r.imag.reshape(40, 40), (1, 0)) / 1e-30
            for b in range(8):
                o = ((b & 1) - (a & 1) + 1) + 3 * (((b >> 1) & 1) - ((a >> 1) & 1) + 1) \
                    + 9 * (((b >> 2) & 1) - ((a >> 2) & 1) + 1)
                blk = Je[a * 5:a * 5 + 5, b * 5:b * 5 + 5].copy()
                blk[:, dmask[:, conn[b]]] = 0.0
                out[q, o] += blk
        for f in range(5):
            if dmask[f, n]:
                out[q, :, f, :] = 0.0
                out[q, 13, f, f] = 1.0
    return out


def stencil_to_csr(Sh, nx, ny, nz):
    """Sparse matrix (unknown f of node n at row f Nn + n) from a host stencil;
    also checks that entries reaching outside the grid are exactly zero."""
    Nn = (nx + 1) * (ny + 1) * (nz + 1)
    Sh = Sh.reshape(27, 5, 5, Nn)
    n = np.arange(Nn)
    i, j, k = n % (nx + 1), (n // (nx + 1)) % (ny + 1), n // ((nx + 1) * (ny + 1))
    rows, cols, vals = [], [], []
    for o in range(27):
        ii, jj, kk = i + o % 3 - 1, j + (o // 3) % 3 - 1, k + o // 9 - 1
        inside = (ii >= 0) & (ii <= nx) & (jj >= 0) & (jj <= ny) & (kk >= 0) & (kk <= nz)
        assert not Sh[o][:, :, ~inside].any(), "entry outside the grid"
        m = ii + (nx + 1) * (jj + (ny + 1) * kk)
        for f in range(5):
            for c in range(5):
                rows.append(f * Nn + n[inside])
                cols.append(c * Nn + m[inside])
                vals.append(Sh[o, f, c, inside])
    rows, cols, vals = (np.concatenate(a) for a in (rows, cols, vals))
    return sparse.csr_matrix((vals, (rows, cols)), shape=(5 * Nn, 5 * Nn))
