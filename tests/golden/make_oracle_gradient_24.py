"""Write tests/golden/oracle_gradient_24.txt with the FP64 oracle alone.

Workload: the 96^3 adjoint configuration's generator at 24^3 elements (unit cube,
h = 1/24, Gr = 1e5, Pr = 0.71, flux patch q = 1, smoothed random design of seed
3), solved by the oracle's damped Newton with direct sparse solves (Gr ramped
1e3 -> 1e4 -> 1e5, final tolerance 1e-13 relative), its objective (mean patch
temperature), the adjoint J^T lambda = -dPhi/dx and the sensitivities
dPhi/dgamma.  Stored: Phi, sum of dPhi/dgamma, and dPhi/dgamma at 128 elements
drawn with seed 4 from the design column.

Run: python tests/golden/make_oracle_gradient_24.py   (a few minutes on one core)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import assemble as A  # noqa: E402
from oracle import element as El  # noqa: E402
from oracle import grid as G  # noqa: E402
from oracle import solve as S  # noqa: E402
from paper_1508_04596_gb300 import synth  # noqa: E402

N = 24
GR = 1e5
PR = 0.71


def main(out=os.path.join(HERE, "oracle_gradient_24.txt")):
    t0 = time.time()
    g = G.Grid(N, N, N, 1.0 / N)
    bc = G.BCs(patch_mode=G.PATCH_FLUX, patch_val=1.0)
    m, v = G.dirichlet(g, bc)
    prm = El.Params(1.0 / N, GR, PR, **synth.MATERIAL)
    prob = A.Problem(g, prm, m, v, flux=G.neumann_rhs(g, bc))
    gam = synth.smoothed_random(N, N, N, 1.0 / N, 3)
    x = np.zeros((5, g.Nn))
    for gr, rtol in ((1e3, 1e-3), (1e4, 1e-3), (GR, 1e-13)):
        prob.prm.Gr = gr
        x, its = S.newton(prob, gam, x, rtol=rtol, atol=1e-14)
        print("Gr %.0e: %d Newton steps, %.0f s" % (gr, its, time.time() - t0), flush=True)
    phi, dphi = S.objective(prob, bc, x)
    lam = S.adjoint(prob, x, gam, -dphi)
    sens = S.sensitivity(prob, x, gam, lam)
    col = np.nonzero(synth.design_column(N, N, N, 1.0 / N))[0]
    sample = np.sort(np.random.default_rng(4).choice(col, size=128, replace=False))
    with open(out, "w") as f:
        f.write("# FP64 oracle, 24^3 flux-patch cavity, Gr=1e5, Pr=0.71, design smoothed_random seed 3\n")
        f.write("# written by tests/golden/make_oracle_gradient_24.py (oracle only)\n")
        f.write("phi %.17e\n" % phi)
        f.write("sum_sens %.17e\n" % sens.sum())
        for e in sample:
            f.write("%d %.17e\n" % (e, sens[e]))
    print("done in %.0f s" % (time.time() - t0))


if __name__ == "__main__":
    main()
