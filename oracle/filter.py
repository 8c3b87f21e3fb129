"""PDE (Helmholtz) density filter (oracle; test infrastructure only).

Sec. 3.2: the design field is regularised by a PDE-based density filter
[Lazarov & Sigmund 2011], with a filter radius of 2.5 element sizes (Sec. 6.3,
6.4).  The filter equation is

    -r^2 lap(rho~) + rho~ = rho   in the domain,  d rho~/dn = 0 on its boundary,
    r = R / (2 sqrt 3),

discretised with trilinear nodal rho~ and the element-constant input rho:

    (r^2 K + M) rho~ = T rho,     K_ab = int grad N_a . grad N_b,  M_ab = int N_a N_b,
                                  T_{n,e} = int_e N_n dV,

and the filtered element value is the mean of its eight nodal values (the
element average of rho~ for trilinear fields).  The element matrices are
integrated here with the 2x2x2 Gauss rule (exact for these integrands).  As a
linear map rho -> gamma~ the filter is P = h^-3 T^T (r^2 K + M)^-1 T, which is
symmetric, so the chain rule dPhi/drho = P^T dPhi/dgamma~ = P dPhi/dgamma~.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .element import GPTS, dshape_ref, shape


def element_matrices(h):
    """Q1 stiffness and mass of a cube of edge h by 2x2x2 Gauss."""
    Ke = np.zeros((8, 8))
    Me = np.zeros((8, 8))
    w = (h / 2.0) ** 3
    for g in range(8):
        N = shape(GPTS[g])
        D = dshape_ref(GPTS[g]) * (2.0 / h)
        Ke += w * D @ D.T
        Me += w * np.outer(N, N)
    return Ke, Me


def filter_matrix(g, R):
    """Assembled r^2 K + M (CSR) and T (CSR, Nn x E) for filter radius R."""
    r2 = (R / (2.0 * np.sqrt(3.0))) ** 2
    Ke, Me = element_matrices(g.h)
    Ae = r2 * Ke + Me
    conn = g.connectivity()
    rows = np.repeat(conn, 8, axis=1).ravel()
    cols = np.tile(conn, (1, 8)).ravel()
    A = sp.coo_matrix((np.tile(Ae.ravel(), g.E), (rows, cols)), shape=(g.Nn, g.Nn)).tocsr()
    T = sp.coo_matrix((np.full(8 * g.E, g.h ** 3 / 8.0),
                       (conn.ravel(), np.repeat(np.arange(g.E), 8))),
                      shape=(g.Nn, g.E)).tocsr()
    return A, T


def apply_filter(g, rho, R):
    """gamma~ = P rho for element-constant rho [E]."""
    A, T = filter_matrix(g, R)
    rt = spla.spsolve(A.tocsc(), T @ rho)
    return (T.T @ rt) / g.h ** 3
