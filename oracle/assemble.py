"""Global residual and assembled Jacobian (oracle; test infrastructure only).

R(x, gamma) = sum over elements of the element rows (``element.element_residual``)
plus the patch flux term, with every Dirichlet row replaced by  x - x_D.

J is the exact derivative of the interior rows with respect to the interior
unknowns, assembled from element Jacobians obtained by complex step,
    J_e[:, k] = Im r_e(x_e + i eps e_k) / eps,   eps = 1e-30
(Squire & Trapp 1998; exact to round-off, and independent of any hand-derived
linearisation).  Dirichlet handling (reading): rows of Dirichlet unknowns are
identity rows, and columns of Dirichlet unknowns are removed from the interior
rows, so J = blockdiag(J_II, I).  A Newton iterate that keeps x_D exact loses
nothing by that, and J^T is the consistent adjoint operator.
"""
import numpy as np
import scipy.sparse as sp

from .element import element_residual
from .grid import NF

CS_EPS = 1e-30


def gather(x, conn):
    """x [5, Nn] -> xe [E, 8, 5]."""
    return np.transpose(x[:, conn], (1, 2, 0))


def element_dofs(g, conn):
    """Global unknown index (f * Nn + n) of each element row, shape [E, 40] ordered (a, f)."""
    f = np.arange(NF)
    return (f[None, None, :] * g.Nn + conn[:, :, None]).reshape(conn.shape[0], 8 * NF)


class Problem:
    """Discrete problem: grid, parameters, Dirichlet data, flux term, element sources."""

    def __init__(self, g, prm, dmask, dval, flux=None, se=None, force=None):
        self.g, self.prm = g, prm
        self.dmask, self.dval = dmask, dval
        self.flux = np.zeros((NF, g.Nn)) if flux is None else flux
        self.se = np.zeros(g.E) if se is None else np.asarray(se, float)
        self.force = force
        self.conn = g.connectivity()
        self.origin = g.elem_ijk() * g.h
        self.edofs = element_dofs(g, self.conn)

    def impose(self, x):
        x = np.array(x, dtype=float, copy=True)
        x[self.dmask] = self.dval[self.dmask]
        return x

    def element_rows(self, x, gam, freeze_tau=False):
        return element_residual(gather(x, self.conn), gam, self.prm, se=self.se,
                                origin=self.origin, force=self.force, freeze_tau=freeze_tau)

    def residual(self, x, gam):
        """R(x, gamma) as [5, Nn]."""
        re = self.element_rows(x, gam)
        R = np.zeros(NF * self.g.Nn, dtype=re.dtype)
        np.add.at(R, self.edofs.ravel(), re.reshape(-1))
        R = R.reshape(NF, self.g.Nn) + self.flux
        R[self.dmask] = x[self.dmask] - self.dval[self.dmask]
        return R

    def element_jacobians(self, x, gam, freeze_tau=False, chunk=4096):
        """J_e [E, 40, 40] by complex step, rows and columns ordered (a, f)."""
        xe = gather(x, self.conn)
        E = xe.shape[0]
        Je = np.empty((E, 8 * NF, 8 * NF))
        eye = np.eye(8 * NF).reshape(8 * NF, 8, NF)
        for s in range(0, E, chunk):
            b = slice(s, min(E, s + chunk))
            nb = b.stop - b.start
            xc = (xe[b][:, None, :, :] + 1j * CS_EPS * eye[None]).reshape(nb * 8 * NF, 8, NF)
            rep = lambda a: np.repeat(a[b], 8 * NF, axis=0)
            r = element_residual(xc, rep(np.asarray(gam)), self.prm, se=rep(self.se),
                                 origin=rep(self.origin), force=self.force,
                                 freeze_tau=freeze_tau)
            # r[(e,k)] = column k of J_e
            Je[b] = np.transpose(r.imag.reshape(nb, 8 * NF, 8 * NF), (0, 2, 1)) / CS_EPS
        return Je

    def jacobian(self, x, gam, freeze_tau=False):
        """Assembled J = blockdiag(J_II, I) in CSR."""
        Je = self.element_jacobians(x, gam, freeze_tau=freeze_tau)
        rows = np.repeat(self.edofs, 8 * NF, axis=1).ravel()
        cols = np.tile(self.edofs, (1, 8 * NF)).ravel()
        n = NF * self.g.Nn
        J = sp.coo_matrix((Je.ravel(), (rows, cols)), shape=(n, n)).tocsr()
        d = self.dmask.ravel()
        keep = sp.diags((~d).astype(float))
        J = keep @ J @ keep + sp.diags(d.astype(float))
        J.sum_duplicates()
        J.eliminate_zeros()
        return J.tocsr()

    def dR_dgamma_elements(self, x, gam):
        """d r_e / d gamma_e by complex step in gamma, [E, 8, 5]."""
        re = self.element_rows(x, np.asarray(gam, float) + 1j * CS_EPS)
        return re.imag / CS_EPS
