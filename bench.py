#!/usr/bin/env python
"""Benchmark of the matrix-free Jacobian-vector product and of the state +
adjoint solves, on synthetic heat-sink cavity workloads.

Default workload: 192 x 192 x 384 elements (domain 1 x 1 x 2, 71.7M unknowns),
Gr = 1e6, Pr = 0.71, base patch heated by a flux, seeded smoothed random design
(the largest single-GPU configuration).  One timed step is one batch of 16 J v
applications in FP64 at the converged state with 16 seeded random directions
(the linearisation store is formed once per step); the reported value is J v
throughput in GDOF/s (all 5 Nn unknowns per application).  The same run also
times, outside the J v region, the full hot path once per precision: Newton
state solve to 1e-8, adjoint solve to 1e-8 and the element sensitivities,
FP32-mixed against plain FP64 (matrix-free, and with every level's Jacobian
assembled into block stencils), plus the cold mixed state solve; and the
build and product times of the assembled FP64 Jacobian at the J v state.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload NAME] [--prec f64|f32] [--no-solve]
N > 1 runs under torchrun: every rank solves its own copy (replicas; the path
does not shard) and rank 0 prints the line.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

NAPPLY = 16  # J v applications per step
DEFAULT_WORKLOAD = "tall192x192x384_gr1e6"
# Operation counts per element (one +, -, *, / or reciprocal square root = 1
# flop; an FMA = 2), of the element routines in csrc/nc_element.cuh, counted by
# instantiating them with a counting number type (tests/host/element_flop_count.cpp;
# tests/test_element_host.py checks that these figures match it).
FLOPS_PER_ELEM = {"residual": 1794, "jvp": 3076, "jtvp": 3196, "diag": 6085, "sens": 1796,
                  "linearize": 848, "jvp_lin": 2214, "jtvp_lin": 2382}
# ALU peaks (whole GPU) from unit counts and the maximum SM clock: 152 SMs x 128
# FP32 lanes x 2 flop x 2.07 GHz, and 152 SMs x 2 FP64 FMA units x 2 flop x 2.07 GHz
# (1.259 TFLOP/s, the GB300's nominal FP64 rate of 1.25).  nc_fma_probe measures
# what dependent FMA chains reach in the same run, as a check.
SMS, SM_MAX_GHZ = 152, 2.07
ALU_PEAK_TFLOPS = {"f32": SMS * 128 * 2 * SM_MAX_GHZ / 1e3, "f64": SMS * 2 * 2 * SM_MAX_GHZ / 1e3}
PEAK_SOURCE = ("unit counts x max SM clock: 152 SMs x 128 FP32 lanes (2 FP64 FMA units) x 2 flop "
               "x 2.07 GHz; checked live by nc_fma_probe (alu_probe)")
# DRAM traffic of one launch of the headline element kernel, from an ncu capture
# at the benchmark's workload; used only while the kernel sources are the ones
# the capture was taken with (their SHA-256 is recorded beside the figure).
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_elem_lin_cached_tall192x192x384_traffic.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1508_04596_gb300", "csrc", f)
                  for f in ("nc_kernels.cu", "nc_element.cuh", "nc_internal.cuh")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--prec", default="f64", choices=["f64", "f32"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--solve-workload", default=None,
                    help="workload of the state/adjoint design-iteration timing (default: --workload)")
    ap.add_argument("--ops-once", action="store_true",
                    help="one J v and one J^T w in --prec at a random BC-consistent state of "
                         "--workload, nothing else (profiling runs)")
    ap.add_argument("--solve-only", action="store_true",
                    help="only the design-iteration solve block of --workload, printed as JSON")
    ap.add_argument("--jv-only", action="store_true",
                    help="only the timed J v step (profiling runs: no end-to-end, operator, "
                         "assembled or vector measurements)")
    ap.add_argument("--vectors-only", default=None, choices=["f32", "f64", "both"],
                    help="only time the FGMRES orthogonalisation step (the HBM-side kernels) "
                         "and print its JSON (profiling runs)")
    return ap.parse_args()


def dist_init(args):
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    return rank, world


def max_over_ranks(value, device=None):
    """The largest per-rank value (the slowest rank's step time); one rank: itself."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.samples, self.stop_ev = index, [], threading.Event()

    def _run(self):
        while not self.stop_ev.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([s.strip() for s in out.split(",")])
            except Exception:
                pass
            self.stop_ev.wait(0.2)

    def __enter__(self):
        self.t = threading.Thread(target=self._run, daemon=True)
        self.t.start()
        return self

    def __exit__(self, *a):
        self.stop_ev.set()
        self.t.join(timeout=6)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if len(s) > 2 + i and s[2 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "MEASURED_PEAKS.json"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0}, "fallback 6.8 TB/s"


# ---------------------------------------------------------------------------------- ours
def kernel_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic(workload, prec):
    """DRAM bytes (read + write) of one launch of the FP64 J v element kernel,
    from the recorded ncu capture, or None when the capture does not match the
    workload, the precision or the current kernel sources."""
    import re
    if prec != "f64" or not os.path.exists(TRAFFIC_FILE):
        return None, "no capture"
    txt = open(TRAFFIC_FILE).read()
    m_b = re.search(r"traffic_bytes_per_launch:\s*(\d+)", txt)
    m_h = re.search(r"sources_sha256:\s*([0-9a-f]{64})", txt)
    m_w = re.search(r"workload:\s*(\S+)", txt)
    if not (m_b and m_h and m_w) or m_w.group(1) != workload:
        return None, "no capture of this workload"
    if m_h.group(1) != kernel_sources_sha():
        return None, "kernel changed since the capture"
    return int(m_b.group(1)), os.path.relpath(TRAFFIC_FILE, ROOT)


def alu_probe(stream):
    """FP32 and FP64 FMA-chain throughput (nc_fma_probe) in TFLOP/s, best of 3
    timed launches of about 0.1 s each after one warm-up launch."""
    import ctypes
    import torch
    from paper_1508_04596_gb300 import nc
    blocks = 8 * torch.cuda.get_device_properties(0).multi_processor_count
    out = {}
    for prec, dt, iters in (("f32", torch.float32, 1 << 20), ("f64", torch.float64, 1 << 15)):
        buf = torch.empty(blocks * 256, dtype=dt, device="cuda")
        code = nc.NC_FP32 if prec == "f32" else nc.NC_FP64
        sp = ctypes.c_void_p(stream.cuda_stream)
        run = lambda: nc.lib.nc_fma_probe(code, blocks, iters, ctypes.c_void_p(buf.data_ptr()), sp)
        if run() != 0:
            raise RuntimeError("nc_fma_probe failed")
        best = float("inf")
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run()
            b.record(stream)
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        if not bool(torch.isfinite(buf).all()):
            raise RuntimeError("nc_fma_probe produced non-finite sums")
        tf = 16.0 * iters * blocks * 256 / (best * 1e-3) / 1e12
        out[prec] = {"tflops": round(tf, 3), "ms": round(best, 3),
                     "derived_peak_tflops": round(ALU_PEAK_TFLOPS[prec], 3),
                     "probe_over_derived": round(tf / ALU_PEAK_TFLOPS[prec], 4)}
        del buf
    out["kernel"] = "k_fma_chain: 8 independent FMA chains per thread, 8 x SMs blocks of 256"
    return out


def solve_block(workload, dev):
    """The full hot path once per precision, as one design iteration of an
    optimisation run (Sec. 3, Sec. 5.1): the state of the current design is
    solved first (cold start, reported separately) and its adjoint, the design
    takes one synthetic optimiser step, then the timed part runs the Newton
    state solve warm-started from the previous state (to 1e-8), the objective,
    the adjoint solve warm-started from the previous adjoint (to 1e-10) and the
    element sensitivities.  The objective is the mean patch temperature, so the
    patch is heated by a flux (a prescribed patch temperature would make the
    objective constant).  The three modes share one context, which is freed on
    return; the FP64 state (or the mixed one) is returned for the J v step."""
    import torch
    from paper_1508_04596_gb300 import nc, synth
    sw = workload
    solve = {}
    sprob = nc.Problem.from_workload(sw, patch="flux")
    sg0 = torch.tensor(synth.design(sw), dtype=torch.float64, device=dev)
    sg1 = torch.tensor(synth.design_step(sw, synth.design(sw), 77), dtype=torch.float64, device=dev)
    # cold start of the current design (mixed, grid sequencing: the coarser grids of
    # the multigrid hierarchy solved first), the common warm start of all modes
    x0 = torch.zeros(sprob.ndof, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, cinf = sprob.newton_solve_sequenced(sg0, x0, nc.default_opts(mixed=1, ramp_steps=3),
                                           check=False)
    torch.cuda.synchronize()
    solve["cold_state_mixed"] = {"s": round(time.perf_counter() - t0, 4),
                                 "method": "grid sequencing (coarsest grid first), load ramping",
                                 "newton_its": cinf["newton_its"],
                                 "lin_its": cinf["lin_its_total"], "status": cinf["status"],
                                 "coarser_grids": [[lv["dims"], lv["newton_its"], lv["lin_its"]]
                                                   for lv in cinf.get("levels", [])]}
    # the adjoint of the current design (mixed, from zero), the common warm start
    # of the next design's adjoint in every mode
    _, dphi0 = sprob.objective(x0)
    t0 = time.perf_counter()
    lam0, a0inf = sprob.adjoint_solve(x0, sg0, -dphi0, opts=nc.default_opts(mixed=1), check=False)
    torch.cuda.synchronize()
    solve["cold_adjoint_mixed"] = {"s": round(time.perf_counter() - t0, 4),
                                   "lin_its": a0inf["lin_its_total"], "status": a0inf["status"]}
    del dphi0
    xs = {}
    for mode, mixed, assembled in (("mixed", 1, 0), ("fp64", 0, 0), ("fp64_assembled", 0, 1)):
        opts = nc.default_opts(mixed=mixed, assembled=assembled, rtol_newton=1e-8, ramp_steps=3)
        aopts = nc.default_opts(mixed=mixed, assembled=assembled, adjoint_start=1)
        # the first calls of a mode allocate its workspace and load its kernels:
        # one short untimed state and adjoint pass
        wopts = nc.default_opts(mixed=mixed, assembled=assembled, max_newton=1, max_lin=2)
        xw = x0.clone()
        sprob.newton_solve(sg1, xw, wopts, check=False)
        _, dw = sprob.objective(xw)
        lw, _ = sprob.adjoint_solve(xw, sg1, -dw, opts=wopts, check=False)
        sprob.sensitivity(xw, sg1, lw)
        del xw, dw, lw
        xm = x0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, inf = sprob.newton_solve(sg1, xm, opts, check=False)
        torch.cuda.synchronize()
        ts = time.perf_counter() - t0
        phi, dphi = sprob.objective(xm)
        lam = lam0.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lam, ainf = sprob.adjoint_solve(xm, sg1, -dphi, lam=lam, opts=aopts, check=False)
        sens = sprob.sensitivity(xm, sg1, lam)
        torch.cuda.synchronize()
        ta = time.perf_counter() - t0
        xs[mode] = (xm, sens)
        solve[mode] = {"state_s": round(ts, 4), "adjoint_plus_sens_s": round(ta, 4),
                       "design_iteration_s": round(ts + ta, 4),
                       "newton_its": inf["newton_its"], "lin_its": inf["lin_its_total"],
                       "state_status": inf["status"], "adjoint_lin_its": ainf["lin_its_total"],
                       "adjoint_status": ainf["status"],
                       "adjoint_sweeps": ainf["newton_its"],
                       "adjoint_rel_res_start": ainf["res_hist"][0] / max(ainf["res0"], 1e-300),
                       "rel_res_final": inf["res_final"] / max(inf["res0"], 1e-300),
                       "adjoint_rel_res_final": ainf["res_final"] / max(ainf["res0"], 1e-300),
                       "phi": phi}
        del lam, dphi
    free, total = torch.cuda.mem_get_info()
    solve["device_memory_used_gb"] = round((total - free) / 1e9, 1)  # all three modes' workspace
    xa, sa = xs["mixed"]
    xb, sb = xs["fp64"]
    xc, sc = xs["fp64_assembled"]
    rel = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
    solve["mixed_vs_fp64_state_rel"] = rel(xa, xb)
    solve["mixed_vs_fp64_sens_rel"] = rel(sa, sb)
    solve["fp64_assembled_vs_fp64_state_rel"] = rel(xc, xb)
    solve["fp64_assembled_vs_fp64_sens_rel"] = rel(sc, sb)
    solve["speedup_design_iteration"] = round(
        solve["fp64"]["design_iteration_s"] / solve["mixed"]["design_iteration_s"], 3)
    solve["speedup_fp64_assembled_vs_fp64"] = round(
        solve["fp64"]["design_iteration_s"] / solve["fp64_assembled"]["design_iteration_s"], 3)
    solve["speedup_mixed_vs_fp64_assembled"] = round(
        solve["fp64_assembled"]["design_iteration_s"] / solve["mixed"]["design_iteration_s"], 3)
    solve["workload"] = sw
    solve["objective"] = ("thermal compliance f = int s T dV (heat-source block)"
                          if synth.WORKLOADS[sw].get("bcs") == "quarter"
                          else "mean patch temperature, patch heated by a flux q = 1")
    solve["design_step"] = "gamma + 0.02 x box-filtered U[-1,1] in the design column (seed 77)"
    solve["warm_starts"] = "state and adjoint from the previous design's (cold mixed solves)"
    x = (xb if solve["fp64"]["state_status"] == "NC_OK" else xa).clone()
    del xs, xa, xb, xc, sa, sb, sc, sg0, sg1, x0, lam0
    sprob.close()
    del sprob
    torch.cuda.empty_cache()
    return solve, x


def run_ours(args, rank, world):
    import torch
    from paper_1508_04596_gb300 import nc, synth
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda")
    cfg = synth.WORKLOADS[args.workload]
    n = (cfg["nx"], cfg["ny"], cfg["nz"])
    stream = torch.cuda.current_stream()
    extra = {"alu_probe": alu_probe(stream)}

    solve, x = {}, None
    if not args.no_solve:
        sw = args.solve_workload or args.workload
        solve, xs = solve_block(sw, dev)
        if sw == args.workload and synth.WORKLOADS[sw]["patch"] == "flux":
            x = xs  # the converged state of the workload's own problem
        del xs
    prob = nc.Problem.from_workload(args.workload)
    gam64 = torch.tensor(synth.design(args.workload), dtype=torch.float64, device=dev)
    ndof = prob.ndof
    if x is None:
        x = torch.tensor(synth.random_state(*n, 1, (0.5, 0.5, 0.5, 50, 1)).ravel(),
                         dtype=torch.float64, device=dev)
        state = "random BC-consistent state"
    else:
        state = "converged FP64 state of the flux-heated problem (warm design iteration)"
    prob.impose_dirichlet(x)

    # --- J v throughput
    dt = torch.float64 if args.prec == "f64" else torch.float32
    xj, gj = x.to(dt), gam64.to(dt)
    g = torch.Generator(device="cpu").manual_seed(1234)
    V = torch.empty(NAPPLY, ndof, dtype=dt, device=dev)
    for i in range(NAPPLY):
        V[i] = torch.randn(ndof, generator=g, dtype=torch.float64).to(dev, dt)
    out = torch.empty_like(xj)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2

    if args.prec == "f64":
        # a step: linearise at the state once, then NAPPLY products (the use in a
        # Krylov solve); the linearisation is inside the timed region
        def step():
            prob.linearize(xj, gj)
            for i in range(NAPPLY):
                prob.jvp_lin(V[i], out)
    else:
        def step():
            for i in range(NAPPLY):
                prob.jvp(xj, gj, V[i], out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(torch.cuda.current_device()) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    t_step = float(np.sum(ms)) / args.steps
    if world > 1:
        import torch.distributed as dist
        t_step = max_over_ranks(t_step, dev)
        dist.barrier()
    value = world * NAPPLY * ndof / (t_step * 1e-3) / 1e9

    # --- roofline of the dominant kernel (the J v element kernel + owner gather; in FP64
    # the linearisation that the step computes once is counted with it)
    if args.prec == "f64":
        flops = (FLOPS_PER_ELEM["jvp_lin"] * NAPPLY + FLOPS_PER_ELEM["linearize"]) * prob.E
    else:
        flops = FLOPS_PER_ELEM["jvp"] * NAPPLY * prob.E
    achieved = flops / (t_step * 1e-3) / 1e12
    peak = ALU_PEAK_TFLOPS[args.prec]
    traffic, traffic_src = recorded_traffic(args.workload, args.prec)
    roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3),
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
            "traffic": traffic, "traffic_source": traffic_src,
            "kernel": ("k_elem_lin_cached<double> + k_gather, k_elem_linearize once per step"
                       if args.prec == "f64" else "k_elem_lin<float> + k_gather"),
            "achieved_over": "the whole step (element kernel, gather and linearisation)",
            "peak_source": PEAK_SOURCE,
            "peak_probe": extra["alu_probe"][args.prec]["tflops"],
            "frac_of_probe": round(achieved / extra["alu_probe"][args.prec]["tflops"], 4)}

    if args.jv_only:
        line = {"metric": "J·v GDOF/s (profiling run, --jv-only)", "value": round(value, 4),
                "unit": "GDOF/s", "ms_per_step": round(t_step, 4), "dtype": args.prec,
                "config": {"workload": args.workload}, "roofline": roof}
        return line if rank == 0 else None

    # --- end to end through the C ABI with host buffers
    xh = xj.cpu().pin_memory()
    gh = gj.cpu().pin_memory()
    Vh = torch.empty((NAPPLY, ndof), dtype=dt).pin_memory()
    Vh.copy_(V)
    outh = torch.empty((NAPPLY, ndof), dtype=dt).pin_memory()
    xd, gd, Vd, od = torch.empty_like(xj), torch.empty_like(gj), torch.empty_like(V), torch.empty_like(V)

    # Copies overlap the products: the inputs stream in on one copy stream (x and
    # gamma first, then each direction), each product waits only for its own
    # direction, and its result streams out on a second copy stream while the
    # next product runs.  Every step starts after the previous one has finished
    # (its results are on the host), so buffers are reused safely.
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_start = torch.cuda.Event()
    ev_x = torch.cuda.Event()
    ev_in = [torch.cuda.Event() for _ in range(NAPPLY)]
    ev_done = [torch.cuda.Event() for _ in range(NAPPLY)]

    def e2e_step():
        ev_start.record(stream)
        s_in.wait_event(ev_start)
        s_out.wait_event(ev_start)
        with torch.cuda.stream(s_in):
            xd.copy_(xh, non_blocking=True)
            gd.copy_(gh, non_blocking=True)
            ev_x.record(s_in)
            for i in range(NAPPLY):
                Vd[i].copy_(Vh[i], non_blocking=True)
                ev_in[i].record(s_in)
        stream.wait_event(ev_x)
        if args.prec == "f64":
            prob.linearize(xd, gd, stream=stream)
        for i in range(NAPPLY):
            stream.wait_event(ev_in[i])
            if args.prec == "f64":
                prob.jvp_lin(Vd[i], od[i], stream=stream)
            else:
                prob.jvp(xd, gd, Vd[i], od[i], stream=stream)
            ev_done[i].record(stream)
            s_out.wait_event(ev_done[i])
            with torch.cuda.stream(s_out):
                outh[i].copy_(od[i], non_blocking=True)
        stream.wait_stream(s_out)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k2 = max(3, args.steps // 4)
    e0.record(stream)
    for _ in range(k2):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = e0.elapsed_time(e1) / k2
    esz = xj.element_size()
    h2d = (xj.numel() + gj.numel() + V.numel()) * esz
    d2h = V.numel() * esz
    e2e = {"value": round(world * NAPPLY * ndof / (t_e2e * 1e-3) / 1e9, 4), "unit": "GDOF/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
    del xh, gh, Vh, outh, xd, gd, Vd, od

    # --- other operators at the same state (for context)
    ops = {}
    x32, g32, v32 = x.float(), gam64.float(), V[0].float()
    x64, v64 = x.double(), V[0].double()
    o32, o64 = torch.empty_like(x32), torch.empty_like(x64)
    for name, fn in (("residual", lambda: prob.residual(x64, gam64, o64)),
                     ("jvp", lambda: prob.jvp(x64, gam64, v64, o64)),
                     ("jtvp", lambda: prob.jtvp(x64, gam64, v64, o64)),
                     ("diag", lambda: prob.diag(x64, gam64, o64)),
                     ("jvp_f32", lambda: prob.jvp(x32, g32, v32, o32)),
                     ("jtvp_f32", lambda: prob.jtvp(x32, g32, v32, o32)),
                     ("residual_f32", lambda: prob.residual(x32, g32, o32))):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(5):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 5
        base = name.replace("_f32", "")
        pk = ALU_PEAK_TFLOPS["f32"] if name.endswith("_f32") else ALU_PEAK_TFLOPS["f64"]
        ops[name] = {"ms": round(t, 4), "gdofs": round(ndof / t / 1e6, 3),
                     "alu_frac": round(FLOPS_PER_ELEM[base] * prob.E / (t * 1e-3) / 1e12 / pk, 4)}
    extra["operators"] = ops
    del x32, g32, v32, o32, o64
    if args.prec == "f64":
        prob.linearize(x64, gam64)  # leave no stale reference to the step's inputs
    free, _ = torch.cuda.mem_get_info()
    S_bytes = 675 * 8 * prob.Nn
    if free > S_bytes + 2 * 8 * 156 * prob.E + (4 << 30):
        extra["assembled"] = assembled_operator(
            prob, x64, gam64, V.double(), ops["jvp"]["ms"],
            t_step / NAPPLY if args.prec == "f64" else None, stream,
            reps=5 if prob.E < 4_000_000 else 2)
    else:
        extra["assembled"] = {"skipped": "%.0f GB free, %.0f GB needed" % (free / 1e9, S_bytes / 1e9)}
    extra["hbm_kernels"] = hbm_kernels(prob, stream)
    if solve:
        extra["solve"] = solve

    if rank != 0:
        return None
    cpu = cpu_baseline(args.workload) if world == 1 and not args.no_cpu else None
    line = {"metric": "J·v GDOF/s and state+adjoint solve time, FP32-mixed vs FP64 at 1e-8 rel",
            "value": round(value, 4), "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_step, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {"workload": args.workload, "grid": list(n), "dof": ndof,
                       "Gr": cfg["Gr"], "Pr": cfg["Pr"], "jv_per_step": NAPPLY,
                       "jv_state": state,
                       "l2": "inputs larger than L2, and L2 flushed between steps (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single-gpu"},
            "clocks": clk.summary(), "e2e": e2e,
            "gpu_launches": (2 * NAPPLY + (1 if args.prec == "f64" else 0)) * args.steps,
            "roofline": roof, "cpu_baseline": cpu}
    line.update(extra)
    return line


def assembled_operator(prob, x, gam, V, jvp_ms, jvp_lin_ms, stream, reps=5):
    """The assembled FP64 Jacobian (nc_assemble) at the J v state: build time and
    the throughput of its product (nc_stencil_apply, one k_stencil_apply launch),
    against the matrix-free products (jvp_ms: nc_jvp; jvp_lin_ms: the benchmark
    step's time per product, linearisation store included).  Per node the product reads 675 FP64
    coefficients (5,400 B) and does 675 FMAs, so it is bound by the FP64 pipe
    (1,350 flop per 5,480 B = 0.25 flop/B, above the 0.18 flop/B balance point);
    boundary nodes have fewer neighbours, and the counts below are exact."""
    import torch
    S = torch.empty(675 * prob.Nn, dtype=torch.float64, device=x.device)
    out = torch.empty_like(x)
    prob.assemble(x, gam, S)
    prob.stencil_apply(S, V[0], out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        prob.assemble(x, gam, S)
    b.record(stream)
    torch.cuda.synchronize()
    t_build = a.elapsed_time(b) / reps
    a.record(stream)
    for i in range(NAPPLY):
        prob.stencil_apply(S, V[i], out)
    b.record(stream)
    torch.cuda.synchronize()
    t_apply = a.elapsed_time(b) / NAPPLY
    ta = t_apply * 1e-3
    ref = jvp_lin_ms if jvp_lin_ms else jvp_ms
    # (node, neighbour) pairs inside the grid: per axis 3 (n + 1) - 2
    pairs = 1.0
    for m in prob.level_dims(0):
        pairs *= 3 * (m + 1) - 2
    flops = 2.0 * 25 * pairs
    nbytes = 8.0 * 25 * pairs + 80.0 * prob.Nn
    del S
    return {"build_ms": round(t_build, 3), "apply_ms": round(t_apply, 4),
            "gdofs": round(prob.ndof / ta / 1e9, 3),
            "matrix_free_jvp_ms": jvp_ms, "matrix_free_jvp_lin_ms": jvp_lin_ms,
            "alu_frac": round(flops / ta / 1e12 / ALU_PEAK_TFLOPS["f64"], 4),
            "hbm_gbs": round(nbytes / ta / 1e9, 1),
            "break_even_products": (round(t_build / (ref - t_apply), 1)
                                    if ref > t_apply else None),
            "kernel": "k_stencil_apply<double> (one thread per node, 27 x 5 x 5 FMAs)"}


def hbm_kernels(prob, stream, n=5 * 129 ** 3, k=10, reps=10, only=None):
    """HBM roofline of the Krylov vector kernels: one FGMRES orthogonalisation
    step (classical Gram-Schmidt twice, normalisation fused; nc_arnoldi_orth, the
    routine the solvers run every iteration) of a vector of the 128^3 cavity's
    size against k = 10 basis columns, FP64 (outer FGMRES) and FP32 (the
    multigrid smoother's precision).  Algorithmic bytes per call: 4 (k + 1)
    column reads + 2 writes of n elements.  The basis (0.9 GB in FP64) exceeds
    L2.  Each call ends with the host read of its k + 1 coefficients, as in
    FGMRES; that wait is inside the timing."""
    import torch
    from paper_1508_04596_gb300 import nc
    peaks, src = measured_peaks()
    out = {}
    for name, dt in (("arnoldi_orth_f64", torch.float64), ("arnoldi_orth_f32", torch.float32)):
        if only and only not in name:
            continue
        ld = nc.mv_ld(n)
        g = torch.Generator(device="cuda").manual_seed(7)
        V = torch.zeros(k * ld, dtype=dt, device="cuda")
        for i in range(k):  # an orthonormal basis, built by the step itself
            col = torch.randn(n, generator=g, dtype=dt, device="cuda")
            if i:
                prob.arnoldi_orth(V, col, i, ld)
            else:
                col /= col.norm()
            V[i * ld:i * ld + n] = col
        w0 = torch.randn(n, generator=g, dtype=dt, device="cuda")
        w = w0.clone()
        for _ in range(2):
            w.copy_(w0)
            prob.arnoldi_orth(V, w, k, ld)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t = 0.0
        for _ in range(reps):
            w.copy_(w0)
            a.record(stream)
            prob.arnoldi_orth(V, w, k, ld)
            b.record(stream)
            torch.cuda.synchronize()
            t += a.elapsed_time(b)
        t /= reps
        nbytes = (4 * (k + 1) + 2) * n * w.element_size()
        gbs = nbytes / (t * 1e-3) / 1e9
        out[name] = {"ms": round(t, 4), "bytes": int(nbytes), "achieved_gbs": round(gbs, 1),
                     "peak_gbs": peaks["hbm_gbs"], "frac": round(gbs / peaks["hbm_gbs"], 4),
                     "peak_source": src, "n": n, "k": k}
        if dt == torch.float64:
            # (4k + 1) n FMAs: at 1.25 TFLOP/s FP64 this step is bound by the FP64
            # pipe (0.70 ms) before HBM (0.58 ms at 6.8 TB/s)
            tf = 2 * (4 * k + 1) * n / (t * 1e-3) / 1e12
            out[name].update({"bound": "alu", "achieved_tflops": round(tf, 3),
                              "alu_peak_tflops": ALU_PEAK_TFLOPS["f64"],
                              "alu_frac": round(tf / ALU_PEAK_TFLOPS["f64"], 4)})
        else:
            out[name]["bound"] = "hbm"
        del V, w, w0
    return out


# ------------------------------------------------------------------------- CPU oracle
def oracle_sample(workload, layers=4, width=64):
    """A bounded sample of the workload: the corner block of at most width x
    width x layers elements at the bottom of the grid, with the workload's design
    there (the oracle assembles its Jacobian by complex step, about 10 s for
    64 x 64 x 4 elements on one core)."""
    from paper_1508_04596_gb300 import synth
    from tests.helpers import oracle_problem, random_bc_state
    cfg = synth.WORKLOADS[workload]
    nx, ny = min(width, cfg["nx"]), min(width, cfg["ny"])
    nz = min(layers, cfg["nz"])
    prob, _ = oracle_problem(nx, ny, nz, cfg["h"], cfg["Gr"], cfg["Pr"], patch_mode=cfg["patch"],
                             **synth.material(cfg))
    gam = synth.design(workload).reshape(cfg["nz"], cfg["ny"], cfg["nx"])[:nz, :ny, :nx].ravel()
    x = random_bc_state(prob, 5)
    return prob, gam, x


def cpu_baseline(workload, reps=16, newton=True):
    """Oracle J v as an assembled CSR SpMV (scipy, one thread) on a bounded sample,
    plus the oracle's residual evaluation on the same sample and its Newton + sparse
    direct (SuperLU) solve of the 12^3 heated cavity to 1e-10."""
    prob, gam, x = oracle_sample(workload)
    t0 = time.perf_counter()
    prob.residual(x, gam)
    t_res = time.perf_counter() - t0
    t0 = time.perf_counter()
    J = prob.jacobian(x, gam)
    t_asm = time.perf_counter() - t0
    v = np.random.default_rng(0).standard_normal(prob.g.ndof)
    t0 = time.perf_counter()
    for _ in range(reps):
        J @ v
    t = (time.perf_counter() - t0) / reps
    out = {"value": round(prob.g.ndof / t / 1e9, 5), "unit": "GDOF/s", "cores": 1,
           "kind": "oracle",
           "sample": "%dx%dx%d bottom corner block of %s: complex-step CSR assembly %.1f s, then %d SpMV"
                     % (prob.g.nx, prob.g.ny, prob.g.nz, workload, t_asm, reps),
           "residual_gdofs": round(prob.g.ndof / t_res / 1e9, 6),
           "cpu_count": os.cpu_count(),
           "affinity": len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else None}
    if newton:
        from oracle import solve as S
        from paper_1508_04596_gb300 import synth
        from tests.helpers import oracle_problem
        name = "cavity12_gr1e3"
        cfg = synth.WORKLOADS[name]
        p, _ = oracle_problem(cfg["nx"], cfg["ny"], cfg["nz"], cfg["h"], cfg["Gr"], cfg["Pr"])
        t0 = time.perf_counter()
        _, its = S.newton(p, synth.design(name), np.zeros((5, p.g.Nn)), rtol=1e-10)
        out["newton_splu_12cube_s"] = round(time.perf_counter() - t0, 2)
        out["newton_splu_12cube_its"] = int(its)
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    prob, gam, x = oracle_sample(args.workload)
    t0 = time.perf_counter()
    J = prob.jacobian(x, gam)
    t_asm = time.perf_counter() - t0
    rng = np.random.default_rng(1234)
    V = rng.standard_normal((NAPPLY, prob.g.ndof))

    def step():
        for i in range(NAPPLY):
            J @ V[i]

    for _ in range(args.warmup):
        step()
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        ts.append(time.perf_counter() - t0)
    t = float(np.mean(ts))
    value = NAPPLY * prob.g.ndof / t / 1e9
    sample = ("%dx%dx%d bottom corner block of %s (assembly %.1f s, untimed), %d SpMV per step"
              % (prob.g.nx, prob.g.ny, prob.g.nz, args.workload, t_asm, NAPPLY))
    return {"impl": "reference", "metric": "J·v GDOF/s and state+adjoint solve time, FP32-mixed vs FP64 at 1e-8 rel",
            "value": round(value, 5), "unit": "GDOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "jv_per_step": NAPPLY},
            "cpu_baseline": {"value": round(value, 5), "unit": "GDOF/s", "cores": 1,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 5), "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.vectors_only:
        import torch
        from paper_1508_04596_gb300 import nc
        prob = nc.Problem(nc.make_params(2, 2, 2, 0.5, 1e3, 0.71), nc.cavity_bcs())
        only = None if args.vectors_only == "both" else args.vectors_only
        print(json.dumps(hbm_kernels(prob, torch.cuda.current_stream(), only=only)))
        return
    if args.ops_once:
        import torch
        from paper_1508_04596_gb300 import nc, synth
        cfg = synth.WORKLOADS[args.workload]
        dt = torch.float64 if args.prec == "f64" else torch.float32
        prob = nc.Problem.from_workload(args.workload)
        g = torch.tensor(synth.design(args.workload), dtype=dt, device="cuda")
        x = torch.tensor(synth.random_state(cfg["nx"], cfg["ny"], cfg["nz"], 1,
                                            (0.5, 0.5, 0.5, 50, 1)).ravel(), dtype=dt, device="cuda")
        prob.impose_dirichlet(x)
        v = torch.randn(prob.ndof, generator=torch.Generator().manual_seed(3)).to("cuda", dt)
        a, b = prob.jvp(x, g, v), prob.jtvp(x, g, v)
        print(json.dumps({"jvp_norm": float(a.norm()), "jtvp_norm": float(b.norm())}))
        return
    if args.solve_only:
        import torch
        solve, _ = solve_block(args.workload, torch.device("cuda"))
        print(json.dumps(solve))
        return
    rank, world = dist_init(args)
    line = run_reference(args, rank, world) if args.impl == "reference" else run_ours(args, rank, world)
    if rank == 0 and line is not None:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
