"""Topology optimisation loop of the paper (Sec. 3.2-3.3), driven through the C ABI.

    python -m paper_1508_04596_gb300.optimize WORKLOAD [--iters N] [--steps S]
                                                       [--nx NX --ny NY --nz NZ] [--fp64]
                                                       [--checkpoint PATH [--every K]]
                                                       [--resume PATH]

Per design iteration: the PDE density filter of the design variables, the
passive elements reset (solid heat-source block, fluid outside the design
domain), the Newton state solve warm-started from the previous iterate's state
(load ramping on failure, Sec. 5.1), the objective (thermal compliance with a
heat source, else the mean patch temperature), the adjoint solve and the
element sensitivities, the filter's chain rule, the volume constraint and one
MMA update (Sec. 3.2).  The material parameters follow the paper's five-step
continuation (Sec. 3.3):

    q_f     0.881, 8.81, 88.1, 881, 881
    q_alpha 8, 8, 8, 98, 998
    alpha   1e5, 1e5, 1e5, 1e6, 1e7

with the iterations split evenly over the steps (the paper runs 500 or 1000
iterations in total and does not give the split).  Every numerical step runs
in libnc's kernels; this module only orders the calls.

Checkpoint / resume: the run's whole state (design variables, the MMA history
and asymptotes, the last converged state that warm-starts the next Newton
solve, the iteration counter and the objective scaling) is saved with
torch.save every K iterations and at the end; a resumed run continues from it
and, the kernels being deterministic, gives the same iterates bit for bit.
"""
import argparse
import json
import time

import numpy as np
import torch

from . import cavity, nc, synth

CONTINUATION = [dict(q_f=0.881, q_alpha=8.0, alpha_max=1e5),
                dict(q_f=8.81, q_alpha=8.0, alpha_max=1e5),
                dict(q_f=88.1, q_alpha=8.0, alpha_max=1e5),
                dict(q_f=881.0, q_alpha=98.0, alpha_max=1e6),
                dict(q_f=881.0, q_alpha=998.0, alpha_max=1e7)]


def regions(cfg):
    """(active design elements, fixed values of the passive elements)."""
    return cavity.design_regions(cfg["nx"], cfg["ny"], cfg["nz"], cfg["h"],
                                 cfg.get("bcs") == "quarter")


class Optimizer:
    """State of one optimisation run on a workload (names of synth.WORKLOADS,
    with optional size overrides nx, ny, nz, h)."""

    def __init__(self, workload, vf=0.05, move=0.2, mixed=1, state_rtol=1e-4, adjoint_rtol=1e-6,
                 **over):
        cfg = dict(synth.WORKLOADS[workload])
        cfg.update(over)
        self.workload, self.over, self.cfg = workload, over, cfg
        self.vf, self.move, self.mixed = vf, move, mixed
        self.state_rtol, self.adjoint_rtol = state_rtol, adjoint_rtol
        des, fixed = regions(cfg)
        dev = "cuda"
        self.active = torch.tensor(des.astype(np.uint8), device=dev)
        self.fixed = torch.tensor(fixed, dtype=torch.float64, device=dev)
        rho0 = np.where(des, 1.0 - vf, fixed)  # the uniform start at the volume fraction
        self.rho = torch.tensor(rho0, dtype=torch.float64, device=dev)
        self.xold1 = torch.tensor(rho0, dtype=torch.float64, device=dev)
        self.xold2 = torch.tensor(rho0, dtype=torch.float64, device=dev)
        E = self.rho.numel()
        self.low = torch.zeros(E, dtype=torch.float64, device=dev)
        self.upp = torch.ones(E, dtype=torch.float64, device=dev)
        self.k = 0
        self.prob = None
        self.step = -1
        self.x = None
        self.lam = None  # the last adjoint: the next adjoint solve's initial guess
        self.f0_scale = None
        self.schedule = None  # (iters, steps) of the run's continuation schedule

    _TENSORS = ("rho", "xold1", "xold2", "low", "upp", "x", "lam")

    def state_dict(self):
        """Everything a resumed run needs, as host tensors and plain values."""
        d = {k: getattr(self, k).detach().cpu() for k in self._TENSORS if getattr(self, k) is not None}
        d.update(workload=self.workload, over=dict(self.over), vf=self.vf, move=self.move,
                 mixed=self.mixed, state_rtol=self.state_rtol, adjoint_rtol=self.adjoint_rtol,
                 k=self.k, step=self.step, f0_scale=self.f0_scale, schedule=self.schedule)
        return d

    def save(self, path):
        torch.save(self.state_dict(), path)

    @classmethod
    def load(cls, path):
        d = torch.load(path, map_location="cpu", weights_only=True)
        opt = cls(d["workload"], vf=d["vf"], move=d["move"], mixed=d["mixed"],
                  state_rtol=d["state_rtol"], adjoint_rtol=d["adjoint_rtol"], **d["over"])
        for k in cls._TENSORS:
            if k in d:
                setattr(opt, k, d[k].to("cuda"))
        opt.k, opt.f0_scale = d["k"], d["f0_scale"]
        opt.schedule = tuple(d["schedule"]) if d.get("schedule") else None
        if d["step"] >= 0:
            x = opt.x
            opt.set_step(d["step"])
            opt.x = x
        return opt

    def set_step(self, step):
        """Material parameters of continuation step `step` (a new context; the
        state and the MMA history carry over)."""
        if step == self.step:
            return
        kw = dict(self.over)
        kw.update(CONTINUATION[step])
        if self.cfg.get("bcs") != "quarter":
            kw["patch"] = "flux"
        self.prob = nc.Problem.from_workload(self.workload, **kw)
        if self.x is None:
            self.x = torch.zeros(self.prob.ndof, dtype=torch.float64, device="cuda")
        self.step = step

    def physical(self):
        """Filtered design, clamped to [0, 1], passive elements reset."""
        g = self.prob.filter(self.rho)
        return self.prob.design_map(g, self.active, self.fixed, 0.0, 1.0, out=g)

    def iterate(self):
        """One design iteration; returns its report."""
        p = self.prob
        t0 = time.perf_counter()
        gam = self.physical()
        sopts = nc.default_opts(mixed=self.mixed, rtol_newton=self.state_rtol, ramp_steps=3)
        _, sinf = p.newton_solve(gam, self.x, sopts, check=False)
        phi, dphi = p.objective(self.x)
        aopts = nc.default_opts(mixed=self.mixed, rtol_adjoint=self.adjoint_rtol,
                                adjoint_start=int(self.lam is not None))
        lam, ainf = p.adjoint_solve(self.x, gam, -dphi, lam=self.lam, opts=aopts, check=False)
        self.lam = lam
        sens = p.sensitivity(self.x, gam, lam)
        # chain rule of the filter (symmetric) on the design variables only
        dfdrho = p.filter(p.design_map(sens, self.active, out=sens))
        dg = torch.empty_like(gam)
        g = p.volume(gam, self.active, self.vf, grad=dg)
        dgdrho = p.filter(dg)
        if self.f0_scale is None:
            self.f0_scale = 1.0 / max(abs(phi), 1e-300)
        lam_v, change = p.mma_update(self.k, self.rho, self.xold1, self.xold2, self.low,
                                     self.upp, dfdrho, g, dgdrho, active=self.active,
                                     move=self.move, df0_scale=self.f0_scale)
        self.k += 1
        torch.cuda.synchronize()
        return {"iter": self.k, "step": self.step, "phi": phi, "g": g, "change": change,
                "multiplier": lam_v, "newton_its": sinf["newton_its"],
                "lin_its": sinf["lin_its_total"], "state_status": sinf["status"],
                "adjoint_lin_its": ainf["lin_its_total"], "adjoint_status": ainf["status"],
                "s": round(time.perf_counter() - t0, 4)}


def run(workload, iters, steps=5, log=print, checkpoint=None, every=10, resume=None,
        stop_after=None, **kw):
    """`iters` design iterations in total over the first `steps` continuation
    steps; with `resume`, continue the run saved there (its iterations count
    towards `iters`); with `checkpoint`, save the run there every `every`
    iterations and at the end; with `stop_after`, stop once that many iterations
    are done in total (the schedule is still the one of `iters` and `steps`, so
    the run can be split over several jobs and resumed)."""
    opt = Optimizer.load(resume) if resume else Optimizer(workload, **kw)
    # the continuation step of iteration k depends on iters and steps: a resumed
    # run must use the schedule it was saved with, or it would jump to another step
    if opt.schedule is not None and opt.schedule != (iters, steps):
        raise ValueError("the run in %s was saved with iters=%d, steps=%d; resume it with the same "
                         "values (got iters=%d, steps=%d)" % ((resume,) + opt.schedule + (iters, steps)))
    opt.schedule = (iters, steps)
    per = max(1, iters // steps)
    end = iters if stop_after is None else min(iters, stop_after)
    hist = []
    while opt.k < end:
        opt.set_step(min(opt.k // per, steps - 1, len(CONTINUATION) - 1))
        r = opt.iterate()
        hist.append(r)
        if log:
            log(json.dumps(r))
        if checkpoint and (opt.k % every == 0 or opt.k == end):
            opt.save(checkpoint)
    return opt, hist


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload")
    ap.add_argument("--iters", type=int, default=25)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--nx", type=int)
    ap.add_argument("--ny", type=int)
    ap.add_argument("--nz", type=int)
    ap.add_argument("--fp64", action="store_true")
    ap.add_argument("--checkpoint", help="save the run here (every --every iterations and at the end)")
    ap.add_argument("--every", type=int, default=10)
    ap.add_argument("--resume", help="continue the run saved in this file")
    ap.add_argument("--stop-after", type=int, help="stop after this many iterations in total "
                    "(with --checkpoint, to resume later with the same --iters and --steps)")
    a = ap.parse_args(argv)
    over = {}
    if a.nx:
        cfg = synth.WORKLOADS[a.workload]
        over = dict(nx=a.nx, ny=a.ny or a.nx, nz=a.nz or a.nx)
        over["h"] = cfg["h"] * cfg["nz"] / over["nz"]
    run(a.workload, a.iters, a.steps, checkpoint=a.checkpoint, every=a.every, resume=a.resume,
        stop_after=a.stop_after, mixed=0 if a.fp64 else 1, **over)


if __name__ == "__main__":
    main()
