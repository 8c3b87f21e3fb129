"""Multigrid transfers and the Galerkin coarse operator (oracle; test
infrastructure only).

Sec. 5.2 preconditions F-GMRES with a geometric multigrid whose coarse
operators are Galerkin projections.  Plain definitions used here:

* Prolongation P (coarse grid of half the elements per axis, nodes 2I on the
  fine grid): trilinear interpolation, the weight of coarse node I at fine node
  i is the product over the axes of 1 (i = 2I), 1/2 (|i - 2I| = 1), else 0,
  applied to each of the 5 fields; rows of fine Dirichlet unknowns are zero
  (they stay at zero) and columns of coarse Dirichlet unknowns are zero.
* Restriction P^T, its transpose.
* Galerkin coarse operator A_c = P^T A_f P with the coarse Dirichlet rows made
  identity rows (the blockdiag(A_II, I) convention of the fine operator).
Unknowns are ordered field-major, f * Nn + node.
"""
import numpy as np
import scipy.sparse as sp

from .grid import Grid, NF


def coarse_grid(g):
    return Grid(g.nx // 2, g.ny // 2, g.nz // 2, 2.0 * g.h)


def prolongation(gf, gc, dmask_f, dmask_c):
    """P [NF*Nn_f, NF*Nn_c] in CSR; dmask_* are [NF, Nn] Dirichlet masks."""
    fi = gf.node_ijk()
    rows, cols, vals = [], [], []
    for ci, I in enumerate(gc.node_ijk()):
        w = np.ones(len(fi))
        for a in range(3):
            d = np.abs(fi[:, a] - 2 * I[a])
            w *= np.where(d == 0, 1.0, np.where(d == 1, 0.5, 0.0))
        nz = np.nonzero(w)[0]
        for f in range(NF):
            rows.append(f * gf.Nn + nz)
            cols.append(np.full(len(nz), f * gc.Nn + ci))
            vals.append(w[nz])
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(NF * gf.Nn, NF * gc.Nn)).tocsr()
    keep_f = sp.diags((~dmask_f.ravel()).astype(float))
    keep_c = sp.diags((~dmask_c.ravel()).astype(float))
    return (keep_f @ P @ keep_c).tocsr()


def galerkin(A_f, P, dmask_c):
    """P^T A_f P with identity rows on the coarse Dirichlet unknowns."""
    d = dmask_c.ravel()
    keep = sp.diags((~d).astype(float))
    A = keep @ (P.T @ A_f @ P) @ keep + sp.diags(d.astype(float))
    return A.tocsr()
