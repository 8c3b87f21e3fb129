"""Element residual of the stabilised equal-order hexahedral discretisation (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

What it computes, term by term, with its source in the paper:

* Strong equations, Sec. 2 Eq. (1a-c): steady incompressible Navier-Stokes with
  the symmetric-gradient viscous term scaled by Pr, Brinkman friction alpha(x) u,
  Boussinesq buoyancy  Gr Pr^2 e^g T, continuity, and convection-diffusion of T
  with conductivity K(x) and source s(x).
* Interpolations, Sec. 3.1 Eq. (7)-(8):
      K(g)     = (g (Ck (1+qf) - 1) + 1) / (Ck (1 + qf g))
      alpha(g) = alpha_max (1 - g) / (1 + qa g)
  with g = 1 fluid, g = 0 solid, element-constant (Sec. 4).
* Stabilisation, App. B: one tau for SUPG and PSPG,
      tau = (tau1^-2 + tau2^-2 + tau3^-2)^(-1/2),
      tau1 = 4 h / ||u_e||_2,  tau2 = h^2 / (4 Pr),  tau3 = 1 / alpha_e,
  ||u_e||_2 the 2-norm of the element's 24 velocity unknowns; the thermal
  tau_T uses tau1 and h^2/(4 K_e) (App. B, last paragraph: "similar
  definitions"; reading: no reaction limit in the energy equation).
* Weak form (reading; the paper defers it to [Alexandersen2014]): with strong
  residuals (second derivatives dropped for trilinear elements)
      rM_i = u_j d_j u_i + d_i p + alpha u_i + Gr Pr^2 e^g_i T - fM_i
      rT   = u_j d_j T - s - fT
  the element rows are
      momentum (a,i): int N_a (u_j d_j u_i + alpha u_i + Gr Pr^2 e^g_i T - fM_i)
                        + Pr d_j N_a (d_j u_i + d_i u_j) - p d_i N_a
                        + tau (u_j d_j N_a) rM_i
      continuity a:   int N_a (d_j u_j - fC) + tau d_i N_a rM_i
      energy a:       int N_a rT + K d_j N_a d_j T + tau_T (u_j d_j N_a) rT
  i.e.  r_{a,f} = sum_g w_g [ N_a f0_f + d_j N_a F1_{f,j} ]  with
      f0_M = u.grad u + alpha u + Gr Pr^2 e^g T - fM,
      F1_M[i,j] = Pr (G_ij + G_ji) - p delta_ij + tau u_j rM_i,
      f0_C = div u - fC,   F1_C[j] = tau rM_j,
      f0_T = rT,           F1_T[j] = K d_j T + tau_T u_j rT.
  fM, fC, fT are manufactured-solution body forces (zero in the method itself).
* Quadrature: 2x2x2 Gauss, points +-1/sqrt(3), weight (h/2)^3 each.

The routine accepts complex arrays so that complex-step derivatives are exact:
tau depends on u only through u_e^T u_e (no conjugation), which is analytic.
"""
import numpy as np

GAUSS = 1.0 / np.sqrt(3.0)
# local node a = ia + 2 ja + 4 ka sits at reference corner (2ia-1, 2ja-1, 2ka-1)
CORNER = np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1]
                   for a in range(8)], dtype=float)
GPTS = CORNER * GAUSS  # the 8 Gauss points, same ordering as the corners


class Params:
    def __init__(self, h, Gr, Pr, alpha_max=1e4, q_alpha=1.0, q_f=1.0, Ck=0.1,
                 g_dir=(0.0, 0.0, -1.0)):
        self.h, self.Gr, self.Pr = float(h), float(Gr), float(Pr)
        self.alpha_max, self.q_alpha, self.q_f, self.Ck = (
            float(alpha_max), float(q_alpha), float(q_f), float(Ck))
        self.g_dir = np.array(g_dir, dtype=float)


def alpha_of(gam, prm):
    """Sec. 3.1 Eq. (8): Brinkman impermeability."""
    return prm.alpha_max * (1.0 - gam) / (1.0 + prm.q_alpha * gam)


def K_of(gam, prm):
    """Sec. 3.1 Eq. (7): effective conductivity."""
    return (gam * (prm.Ck * (1.0 + prm.q_f) - 1.0) + 1.0) / (prm.Ck * (1.0 + prm.q_f * gam))


def shape(xi):
    """Trilinear shape functions N_a(xi), shape [8]."""
    return np.prod((1.0 + CORNER * xi[None, :]) / 2.0, axis=1)


def dshape_ref(xi):
    """dN_a/dxi_d on the reference cube, shape [8, 3]."""
    f = (1.0 + CORNER * xi[None, :]) / 2.0
    out = np.empty((8, 3))
    for d in range(3):
        others = [o for o in range(3) if o != d]
        out[:, d] = CORNER[:, d] / 2.0 * f[:, others[0]] * f[:, others[1]]
    return out


def tau_momentum(S, alpha, prm):
    """App. B: tau = (tau1^-2 + tau2^-2 + tau3^-2)^(-1/2) with S = u_e^T u_e."""
    h = prm.h
    inv_t1sq = S / (4.0 * h) ** 2          # tau1 = 4h/sqrt(S)
    inv_t2sq = (4.0 * prm.Pr / h ** 2) ** 2  # tau2 = h^2/(4 Pr)
    inv_t3sq = alpha ** 2                  # tau3 = 1/alpha
    return (inv_t1sq + inv_t2sq + inv_t3sq) ** -0.5


def tau_energy(S, K, prm):
    """Thermal SUPG parameter: tau1 as above, tau2 with K_e in place of Pr."""
    h = prm.h
    return (S / (4.0 * h) ** 2 + (4.0 * K / h ** 2) ** 2) ** -0.5


def element_residual(xe, gam, prm, se=None, origin=None, force=None, freeze_tau=False):
    """Element residual vectors.

    xe     [B, 8, 5] nodal unknowns (u, v, w, p, T) of B elements (real or complex)
    gam    [B] element design values
    se     [B] element heat source s_e (default 0)
    origin [B, 3] physical coordinates of local node 0 (only needed with ``force``)
    force  optional callable xyz[B,3] -> (fM[B,3], fC[B], fT[B]) body forces
    freeze_tau  evaluate tau, tau_T at the real part of the state, so that
           complex-step derivatives leave out dtau/du (the inconsistent
           Jacobian that App. B compares against)
    Returns r [B, 8, 5].
    """
    B = xe.shape[0]
    h = prm.h
    dt = np.result_type(xe.dtype, np.asarray(gam).dtype, float)
    gam = np.asarray(gam)
    se = np.zeros(B) if se is None else np.asarray(se)
    alpha = alpha_of(gam, prm)
    K = K_of(gam, prm)
    ue = xe[:, :, 0:3]
    S = np.sum(ue * ue, axis=(1, 2))   # u_e^T u_e, no conjugation
    if freeze_tau:
        S = np.real(S)
    tau = tau_momentum(S, alpha, prm)
    tauT = tau_energy(S, K, prm)
    beta = prm.Gr * prm.Pr ** 2
    eg = prm.g_dir
    w = (h / 2.0) ** 3
    r = np.zeros((B, 8, 5), dtype=dt)
    for g in range(8):
        N = shape(GPTS[g])                 # [8]
        D = dshape_ref(GPTS[g]) * (2.0 / h)  # [8, 3] physical gradients
        u = np.einsum("a,bai->bi", N, ue)
        G = np.einsum("aj,bai->bij", D, ue)    # G[i,j] = d_j u_i
        p = np.einsum("a,ba->b", N, xe[:, :, 3])
        gp = np.einsum("aj,ba->bj", D, xe[:, :, 3])
        T = np.einsum("a,ba->b", N, xe[:, :, 4])
        gT = np.einsum("aj,ba->bj", D, xe[:, :, 4])
        if force is not None:
            xyz = origin + (GPTS[g] + 1.0) * (h / 2.0)
            fM, fC, fT = force(xyz)
        else:
            fM, fC, fT = 0.0, 0.0, 0.0
        conv = np.einsum("bj,bij->bi", u, G)     # u_j d_j u_i
        body = alpha[:, None] * u + beta * eg[None, :] * T[:, None] - fM
        rM = conv + gp + body
        rT = np.einsum("bj,bj->b", u, gT) - se - fT
        f0M = conv + body
        F1M = prm.Pr * (G + np.swapaxes(G, 1, 2)) - p[:, None, None] * np.eye(3)[None] \
            + tau[:, None, None] * rM[:, :, None] * u[:, None, :]
        f0C = np.einsum("bii->b", G) - fC
        F1C = tau[:, None] * rM
        f0T = rT
        F1T = K[:, None] * gT + tauT[:, None] * u * rT[:, None]
        r[:, :, 0:3] += w * (N[None, :, None] * f0M[:, None, :]
                             + np.einsum("aj,bij->bai", D, F1M))
        r[:, :, 3] += w * (N[None, :] * f0C[:, None] + np.einsum("aj,bj->ba", D, F1C))
        r[:, :, 4] += w * (N[None, :] * f0T[:, None] + np.einsum("aj,bj->ba", D, F1T))
    return r


def dtau_du_printed(ue, alpha, prm):
    """App. B, printed derivative:
    dtau/du_e = -tau (1 + (tau1/tau2)^2 + (tau1/tau3)^2)^-1 (u_e^T u_e)^-1 u_e^T.
    ue [24] (one element), returns [24]."""
    S = ue @ ue
    tau = tau_momentum(S, alpha, prm)
    t1 = 4.0 * prm.h / np.sqrt(S)
    t2 = prm.h ** 2 / (4.0 * prm.Pr)
    t3 = 1.0 / alpha
    return -tau / (1.0 + (t1 / t2) ** 2 + (t1 / t3) ** 2) / S * ue


def dtau_dgamma_printed(ue, gam, prm):
    """App. B, printed derivative:
    dtau/dgamma_e = -(tau/tau3) ((tau3/tau1)^2 + (tau3/tau2)^2 + 1)^-1 dalpha_e/dgamma_e."""
    S = ue @ ue
    alpha = alpha_of(gam, prm)
    tau = tau_momentum(S, alpha, prm)
    t1 = 4.0 * prm.h / np.sqrt(S)
    t2 = prm.h ** 2 / (4.0 * prm.Pr)
    t3 = 1.0 / alpha
    dalpha = -prm.alpha_max * (1.0 + prm.q_alpha) / (1.0 + prm.q_alpha * gam) ** 2
    return -(tau / t3) / ((t3 / t1) ** 2 + (t3 / t2) ** 2 + 1.0) * dalpha
