"""Method of moving asymptotes for one inequality constraint (oracle; test
infrastructure only).

The paper solves its optimisation problem (Sec. 3.2: minimise the thermal
compliance subject to the volume constraint g(gamma) = int_{Omega_d} (1 - gamma) dV
<= v_f |Omega_d| and 0 <= gamma <= 1) with MMA [Svanberg 1987] and prints none of
its details.  Reading used here (Svanberg's method as commonly stated):

* Asymptotes.  Iterations k = 0, 1: L = x - s0 (xmax - xmin), U = x + s0 (xmax - xmin)
  with s0 = 0.5.  From k = 2: with sign_j = (x^k - x^{k-1})(x^{k-1} - x^{k-2}) the
  factor is 0.7 if sign_j < 0 (oscillation), 1.2 if sign_j > 0, else 1;
  L = x - factor (x^{k-1} - L^{k-1}), U = x + factor (U^{k-1} - x^{k-1}), then
  L is kept in [x - 10 d, x - 0.01 d] and U in [x + 0.01 d, x + 10 d], d = xmax - xmin.
* Move limits.  alpha = max(xmin, L + 0.1 (x - L), x - move d),
  beta = min(xmax, U - 0.1 (U - x), x + move d).
* Convex approximation of f_i (i = 0 objective, 1 constraint) with
  a = df_i/dx_j:  p_ij = (U - x)^2 (1.001 a+ + 0.001 a- + 1e-5 / d),
  q_ij = (x - L)^2 (0.001 a+ + 1.001 a- + 1e-5 / d)  (a+ = max(a, 0), a- = max(-a, 0)),
  f~_i(y) = f_i(x) + sum_j [p_ij (1/(U - y) - 1/(U - x)) + q_ij (1/(y - L) - 1/(x - L))].
* Subproblem min f~_0 s.t. f~_1 <= 0, alpha <= y <= beta, by its dual: for a
  multiplier lam >= 0 the Lagrangian separates and its minimiser per variable
  is y_j = (L sqrt(P) + U sqrt(Q)) / (sqrt(P) + sqrt(Q)) clipped to [alpha, beta],
  P = p_0j + lam p_1j, Q = q_0j + lam q_1j.  f~_1(y(lam)) does not increase with
  lam: lam = 0 if f~_1(y(0)) <= 0, else lam brackets by doubling from 1 and
  bisects until f~_1(y(lam)) = 0 (the constraint is active).
"""
import numpy as np

S0, INCR, DECR = 0.5, 1.2, 0.7
RAA0 = 1e-5


def volume_constraint(gam, active, vf, h=1.0):
    """The volume constraint of Sec. 3.2 normalised by the allowed volume:
    g = int_{Omega_d} (1 - gamma) dV / (v_f |Omega_d|) - 1  (<= 0 when satisfied),
    gamma element-constant on cubes of edge h, Omega_d the active (design)
    elements (all when active is None).  Returns g and dg/dgamma_e (0 on
    inactive elements)."""
    gam = np.asarray(gam, dtype=float)
    act = np.ones(gam.shape, bool) if active is None else np.asarray(active, bool)
    vol_d = h ** 3 * act.sum()
    g = h ** 3 * np.sum(1.0 - gam[act]) / (vf * vol_d) - 1.0
    return g, np.where(act, -h ** 3 / (vf * vol_d), 0.0)


def asymptotes(k, x, xold1, xold2, low, upp, xmin, xmax):
    """Asymptotes for iteration k (0-based) from the two previous iterates and
    the previous asymptotes."""
    d = xmax - xmin
    if k < 2:
        return x - S0 * d, x + S0 * d
    sgn = (x - xold1) * (xold1 - xold2)
    fac = np.where(sgn < 0, DECR, np.where(sgn > 0, INCR, 1.0))
    low = x - fac * (xold1 - low)
    upp = x + fac * (upp - xold1)
    low = np.clip(low, x - 10.0 * d, x - 0.01 * d)
    upp = np.clip(upp, x + 0.01 * d, x + 10.0 * d)
    return low, upp


def bounds(x, low, upp, xmin, xmax, move):
    d = xmax - xmin
    alpha = np.maximum.reduce([np.full_like(x, xmin), low + 0.1 * (x - low), x - move * d])
    beta = np.minimum.reduce([np.full_like(x, xmax), upp - 0.1 * (upp - x), x + move * d])
    return alpha, beta


def approx_coefficients(x, low, upp, df, d):
    """p, q of the convex approximation of one function with gradient df."""
    ap, am = np.maximum(df, 0.0), np.maximum(-df, 0.0)
    p = (upp - x) ** 2 * (1.001 * ap + 0.001 * am + RAA0 / d)
    q = (x - low) ** 2 * (0.001 * ap + 1.001 * am + RAA0 / d)
    return p, q


def approx_value(f, x, y, low, upp, p, q):
    return f + np.sum(p * (1.0 / (upp - y) - 1.0 / (upp - x)) + q * (1.0 / (y - low) - 1.0 / (x - low)))


def y_of_lambda(lam, low, upp, alpha, beta, p0, q0, p1, q1):
    P, Q = p0 + lam * p1, q0 + lam * q1
    sP, sQ = np.sqrt(P), np.sqrt(Q)
    return np.clip((low * sP + upp * sQ) / (sP + sQ), alpha, beta)


def mma_step(k, x, xold1, xold2, low, upp, f1, df0, df1, xmin=0.0, xmax=1.0, move=0.2,
             bisect_steps=200):
    """One MMA iteration.  Returns (x_new, low, upp, lam)."""
    d = xmax - xmin
    low, upp = asymptotes(k, x, xold1, xold2, low, upp, xmin, xmax)
    alpha, beta = bounds(x, low, upp, xmin, xmax, move)
    p0, q0 = approx_coefficients(x, low, upp, df0, d)
    p1, q1 = approx_coefficients(x, low, upp, df1, d)

    def g(lam):
        y = y_of_lambda(lam, low, upp, alpha, beta, p0, q0, p1, q1)
        return approx_value(f1, x, y, low, upp, p1, q1), y

    g0, y = g(0.0)
    if g0 <= 0.0:
        return y, low, upp, 0.0
    hi = 1.0
    for _ in range(bisect_steps):
        if g(hi)[0] <= 0.0:
            break
        hi *= 2.0
    lo = 0.0
    for _ in range(bisect_steps):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if g(mid)[0] > 0.0:
            lo = mid
        else:
            hi = mid
    lam = hi
    return g(lam)[1], low, upp, lam
