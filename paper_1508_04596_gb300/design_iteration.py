"""One design iteration of an optimisation run, for timing and profiling.

    python -m paper_1508_04596_gb300.design_iteration WORKLOAD [--fp64] [--no-adjoint] [--galerkin]
                                                      [--assembled] [--restart M] [--sequence]
                                                      [--cold-adjoint]

Solves the state and the adjoint of the workload's design from a cold start,
takes one synthetic optimiser step of the design (``synth.design_step``), then
runs the Newton state solve warm-started from the previous state, the
objective, the adjoint solve warm-started from the previous adjoint (from zero
with --cold-adjoint) and the element sensitivities (Sec. 3.2, Sec. 5) inside an
NVTX range named "warm", so that a profiler can be restricted to it
(``ncu --nvtx --nvtx-include warm/``).
Prints the iteration counts and wall times of the warm part.  With --galerkin the
warm solves use Galerkin coarse operators (P^T A P) instead of rediscretised ones.
"""
import argparse
import json
import time

import torch

from . import nc, synth


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--fp64", action="store_true", help="plain FP64 instead of mixed precision")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--galerkin", action="store_true", help="Galerkin coarse operators")
    ap.add_argument("--assembled", action="store_true",
                    help="assemble every level's Jacobian into a block stencil")
    ap.add_argument("--restart", type=int, default=30, help="FGMRES restart (memory: 2 vectors each)")
    ap.add_argument("--sequence", action="store_true",
                    help="cold start by grid sequencing (solve the coarser grids first)")
    ap.add_argument("--cold-adjoint", action="store_true",
                    help="start the warm iteration's adjoint from zero, not the previous adjoint")
    a = ap.parse_args(argv)
    mixed = 0 if a.fp64 else 1
    prob = nc.Problem.from_workload(a.workload, patch="flux")
    gh = synth.design(a.workload)
    g0 = torch.tensor(gh, dtype=torch.float64, device="cuda")
    g1 = torch.tensor(synth.design_step(a.workload, gh, 77), dtype=torch.float64, device="cuda")
    del gh
    x = torch.zeros(prob.ndof, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    copts = nc.default_opts(mixed=1, ramp_steps=3, restart=a.restart)
    if a.sequence:
        _, cinf = prob.newton_solve_sequenced(g0, x, copts)
    else:
        _, cinf = prob.newton_solve(g0, x, copts)
    torch.cuda.synchronize()
    cold = {"cold_state_s": time.perf_counter() - t0, "cold_newton_its": cinf["newton_its"],
            "cold_lin_its": cinf["lin_its_total"], "cold_levels": cinf.get("levels"),
            "cold_res_hist": cinf["res_hist"]}
    lam = None
    if not a.no_adjoint and not a.cold_adjoint:  # the previous design's adjoint
        _, d0 = prob.objective(x)
        lam, a0 = prob.adjoint_solve(x, g0, -d0, opts=nc.default_opts(mixed=1, restart=a.restart))
        cold["cold_adjoint_lin_its"] = a0["lin_its_total"]
        del d0
    # load the kernels and allocate the workspace of this precision (untimed)
    gal = 1 if a.galerkin else 0
    asm = 1 if a.assembled else 0
    kw = dict(mixed=mixed, galerkin=gal, assembled=asm, restart=a.restart)
    wopts = nc.default_opts(max_newton=1, max_lin=2, **kw)
    xw = x.clone()
    prob.newton_solve(g1, xw, wopts, check=False)
    _, dw = prob.objective(xw)
    lw, _ = prob.adjoint_solve(xw, g1, -dw, opts=wopts, check=False)
    prob.sensitivity(xw, g1, lw)
    del xw, dw, lw
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("warm")
    t0 = time.perf_counter()
    _, inf = prob.newton_solve(g1, x, nc.default_opts(**kw), check=False)
    torch.cuda.synchronize()
    out = {"workload": a.workload, "mixed": mixed, "galerkin": gal, "assembled": asm,
           "state_s": time.perf_counter() - t0, "newton_its": inf["newton_its"],
           "lin_its": inf["lin_its_total"], "state_status": inf["status"],
           "state_res_hist": inf["res_hist"]}
    if not a.no_adjoint:
        t0 = time.perf_counter()
        phi, dphi = prob.objective(x)
        lam, ainf = prob.adjoint_solve(x, g1, -dphi, lam=lam,
                                       opts=nc.default_opts(adjoint_start=int(lam is not None), **kw),
                                       check=False)
        prob.sensitivity(x, g1, lam)
        torch.cuda.synchronize()
        out.update(adjoint_plus_sens_s=time.perf_counter() - t0, phi=phi,
                   adjoint_lin_its=ainf["lin_its_total"], adjoint_status=ainf["status"])
    torch.cuda.nvtx.range_pop()
    free, total = torch.cuda.mem_get_info()
    out.update(cold, dof=prob.ndof, restart=a.restart,
               device_mem_used_gb=round((total - free) / 1e9, 1))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
