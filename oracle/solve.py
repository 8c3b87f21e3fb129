"""Newton solve, objective, adjoint and sensitivities (oracle; test infrastructure only).

* Damped Newton, Sec. 5.1: the step length minimises a quadratic fitted to the
  L2 norm of the residual at 0, 50 % and 100 % of the Newton step.  Reading of
  the fit: q(l) = a l^2 + b l + c through (0, n0), (1/2, n_half), (1, n1).  If
  a > 0 and the minimiser -b/(2a) lies in (0, 1], the step is that minimiser,
  raised to at least 0.05; otherwise the sampled length (1/2 or 1) with the
  smaller norm, the longer one on a tie.  Linear systems are solved directly
  (sparse LU), so the linear solve is exact.
* Objective.  With a heat source and no patch, the thermal compliance of
  Sec. 3.2, f = int_omega s T dV, with s element-constant and T trilinear:
  int_e N_a dV = h^3/8 exactly.  With a patch (reading of the same objective
  for a heated patch): Phi = (1/|Gamma_p|) int_{Gamma_p} T dA, the mean
  temperature of the bottom patch, 2x2 Gauss per face (exact for bilinear T).
* Adjoint, Sec. 3.2: J^T lambda = -dPhi/dx with J = blockdiag(J_II, I).
* Sensitivities: dPhi/dgamma_e = dPhi/dgamma_e|explicit (zero here)
  + lambda^T dR/dgamma_e, the element rows of Dirichlet unknowns excluded.
"""
import numpy as np
import scipy.sparse.linalg as spla

from .assemble import gather
from .grid import NF, PATCH_NONE, patch_faces


def line_search_length(n0, nh, n1):
    a = 2.0 * (n1 - 2.0 * nh + n0)
    b = n1 - n0 - a
    if a > 0.0:
        lam = -b / (2.0 * a)
        if 0.0 < lam <= 1.0:
            return max(lam, 0.05)
    return 0.5 if nh < n1 else 1.0


def newton(prob, gam, x0, rtol=1e-10, atol=0.0, maxit=50, linsolve=None, history=None):
    """Damped Newton from x0 (Dirichlet values imposed first).  Returns (x, its)."""
    x = prob.impose(x0)
    R = prob.residual(x, gam)
    n0 = r0 = np.linalg.norm(R)
    its = 0
    if history is not None:
        history.append(n0)
    while n0 > max(rtol * r0, atol) and its < maxit:
        J = prob.jacobian(x, gam)
        if linsolve is None:
            d = spla.splu(J.tocsc()).solve(-R.ravel())
        else:
            d = linsolve(J, -R.ravel())
        d = d.reshape(NF, -1)
        Rh = prob.residual(x + 0.5 * d, gam)
        R1 = prob.residual(x + d, gam)
        nh, n1 = np.linalg.norm(Rh), np.linalg.norm(R1)
        lam = line_search_length(n0, nh, n1)
        if lam == 1.0:
            x, R = x + d, R1
        elif lam == 0.5:
            x, R = x + 0.5 * d, Rh
        else:
            x = x + lam * d
            R = prob.residual(x, gam)
        n0 = np.linalg.norm(R)
        its += 1
        if history is not None:
            history.append(n0)
    return x, its


def objective(prob, bc, x):
    """Objective and its gradient dPhi/dx ([5, Nn]): thermal compliance when the
    patch mode is none and a source is present, else the mean patch temperature."""
    g = prob.g
    dphi = np.zeros((NF, g.Nn))
    if bc.patch_mode == PATCH_NONE and np.any(prob.se != 0.0):
        w = prob.se * g.h ** 3 / 8.0
        for a in range(8):
            np.add.at(dphi[4], prob.conn[:, a], w)
        return float(np.sum(dphi * x)), dphi
    faces = patch_faces(g, bc)
    if faces.size == 0:
        return 0.0, dphi
    area = faces.size * g.h * g.h
    conn = prob.conn
    for e in faces:
        for a in range(4):
            dphi[4, conn[e, a]] += g.h * g.h / 4.0 / area
    return float(np.sum(dphi * x)), dphi


def adjoint(prob, x, gam, rhs):
    """Solve J(x)^T lam = rhs directly.  rhs, lam as [5, Nn]."""
    J = prob.jacobian(x, gam)
    return spla.splu(J.T.tocsc()).solve(rhs.ravel()).reshape(NF, -1)


def sensitivity(prob, x, gam, lam):
    """dPhi/dgamma_e = lambda_e^T dr_e/dgamma_e (Dirichlet rows excluded), [E]."""
    lam_int = np.where(prob.dmask, 0.0, lam)
    dre = prob.dR_dgamma_elements(x, gam)
    return np.einsum("eaf,eaf->e", gather(lam_int, prob.conn), dre)


def gram_schmidt_twice(V, w):
    """One orthogonalisation step of the FGMRES Arnoldi process (Sec. 5.2), by its
    plain definition: classical Gram-Schmidt of w against the orthonormal rows
    of V, applied twice.  V: [k, n], w: [n] (FP64).  Returns (h, nu, q) with
    h = h1 + h2 the Hessenberg column, nu = ||w - V^T h|| and q the unit vector
    (w - V^T h) / nu, so that w = V^T h + nu q."""
    h1 = V @ w
    w1 = w - V.T @ h1
    h2 = V @ w1
    w2 = w1 - V.T @ h2
    nu = float(np.linalg.norm(w2))
    return h1 + h2, nu, w2 / nu
