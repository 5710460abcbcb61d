#!/usr/bin/env python
"""Throughput of the FR-SG stage on GB300: DOF-stage updates per second.

A "step" is one SSP-RK3 time step (three fused stage launches: z-evaluation, flux,
Galerkin projection, FR derivative with LLF + Radau correction, SSP combination,
detector and filter) of the stochastic Burgers workload: 1024 elements, P = 3,
N = 8, Q = 16 (36,864 DOF), exponential filter switched by the detector, CFL 0.1.
DOF = elements x solution points x gPC modes x variables; one step is 3 DOF-stages
per DOF.  Both the plain FP64 form and the FP32 form are measured; the line reports
the faster form whose error against the FP64 oracle meets its stated bound.

Timing: W untimed steps, then K steps each bracketed by CUDA events on the solver's
stream, with a 256 MiB memset between timed steps to flush the 129 MB L2 (the state
is 0.3 MB, so every timed step starts from HBM).  Max over ranks under torchrun
(N > 1 runs independent replicas: "weak" scaling, no collective on the data path).

--impl reference times the FP64 CPU oracle (numpy, one core) on the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2112_05946_gb300 import workloads  # noqa: E402

METRIC = "DOF-stage updates/s"
UNIT = "DOF-stage/s"
ERR_BOUND = {"fp64": 1e-12, "fp32": 1e-5}     # relative L2 vs the FP64 oracle after the accuracy run
ACC_STEPS = 50


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="burgers", choices=sorted(workloads.ALL))
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="bounded oracle sample length")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the Sod, 2D, batched and adjoint lines")
    ap.add_argument("--only", default=None, choices=["burgers", "sod", "shock_vortex", "batch", "adjoint"],
                    help="measure one extra workload alone and print its line (for profiling runs)")
    return ap.parse_args(argv)


def max_over_ranks(torch, v, world, device):
    """The largest value over all ranks (the step time the whole job is held to); v itself
    when there is one rank."""
    if world == 1:
        return v
    t = torch.tensor([v], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, dof, stages, ms):
    """DOF-stage updates per second of the whole job: each of the `world` ranks advances its
    own replica of `dof` unknowns through `stages` stages every `ms` milliseconds."""
    return world * dof * stages / (ms * 1e-3)


def load_tune_cache(frsg):
    """Merge the autotuner choices of an earlier run (FRSG_TUNE_CACHE) so that a profiler
    run of the same command times the layouts the plain run chose."""
    path = os.environ.get("FRSG_TUNE_CACHE")
    if path and os.path.exists(path):
        frsg.tune_cache_load(path)
    return path


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_sizes(wl):
    s = wl["solver"]
    n1 = s["P"] + 1
    E = s["nx"] * (s.get("ny", 1) if s.get("dim", 1) == 2 else 1)
    Np = n1 ** s.get("dim", 1)
    M = s["N"] + 1
    S = 1 if s["equation"] != "euler" else (3 if s.get("dim", 1) == 1 else 4)
    return E, Np, M, S


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- our arm

# DRAM bytes per launch of the benchmark's kernels, from ncu captures of the current build
# (dram__bytes_read.sum + dram__bytes_write.sum, one launch, L2 flushed by ncu before it;
# profiles/step1d_fused_burgers_E1024_ncu.md)
# keyed by (kernel, precision, tile): the halo re-reads depend on the tile
MEASURED_TRAFFIC = {("step1d_fused_kernel", "fp32", 7): 177408}


def measure_form(torch, frsg, wl, precision, steps, warmup, stream, flush, oracle_ref):
    E, Np, M, S = workload_sizes(wl)
    dof = E * Np * M * S
    s = frsg.Solver(stream=stream.cuda_stream, precision=precision, **wl["solver"])
    variant, tile = s.autotune()
    x, z = s.nodes()
    u0 = workloads.nodal_values(wl["ic"], x, z)
    dx = (wl["solver"]["x1"] - wl["solver"]["x0"]) / wl["solver"]["nx"]
    dt = wl["cfl"] * dx / wl["lam0"]
    esz = 8 if precision == "fp64" else 4

    # accuracy run against the FP64 oracle
    s.set_initial_nodal(u0)
    s.rk_step(dt, ACC_STEPS, graph=True)
    s.check()
    got = s.get_state()
    err = float(np.linalg.norm(got - oracle_ref) / np.linalg.norm(oracle_ref))

    # throughput: per-step events with an L2 flush between steps
    s.set_initial_nodal(u0)
    with torch.cuda.stream(stream):
        s.rk_step(dt, warmup, graph=True)
        stream.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        l0 = s.launch_count()
        torch.cuda.nvtx.range_push("timed")            # profilers can select the timed launches
        for i in range(steps):
            flush.zero_()
            starts[i].record(stream)
            s.rk_step(dt, 1, graph=True)
            ends[i].record(stream)
        torch.cuda.nvtx.range_pop()
        stream.synchronize()
        launches = s.launch_count() - l0
        step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]

        # kernel durations: the three stage launches timed one by one (same flush)
        kst = min(steps, 200)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(kst)]
        for i in range(kst):
            flush.zero_()
            evs[i][0].record(stream)
            for st in range(3):
                s.stage(st, dt)
                evs[i][st + 1].record(stream)
        stream.synchronize()
        stage_ms = [[evs[i][st].elapsed_time(evs[i][st + 1]) for st in range(3)] for i in range(kst)]

        # steady state: back-to-back graph replays, state resident in L2 (context only)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        s.rk_step(dt, steps, graph=True)
        ev1.record(stream)
        stream.synchronize()
        steady_ms = ev0.elapsed_time(ev1) / steps
    s.check()

    # end to end through the public API with host buffers: pinned host state in, step, state out
    h_in = torch.empty((E, Np, M, S), dtype=torch.float64, pin_memory=True)
    h_in.copy_(torch.from_numpy(got))
    h_out = torch.empty_like(h_in)
    e2e_steps = min(steps, 200)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hi, ho = h_in.numpy(), h_out.numpy()
    for _ in range(e2e_steps):
        s.advance(hi, ho, dt, 1)             # state in, one step, state out: one call, one sync
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    s.close()

    ms = float(np.mean(step_ms))
    mean_stage = np.mean(np.array(stage_ms), axis=0)           # ms per stage launch
    if variant == 3:
        # one launch per step whose stage states stay on chip: it must read u^n and write
        # u^{n+1}, two state arrays per step
        alg_bytes = [2 * esz * dof]
    else:
        arrays = [2, 3, 3]                                     # state arrays read+written per stage
        alg_bytes = [a * esz * dof for a in arrays]
    if variant in (2, 3):
        # one launch per step: the timed step is the kernel
        achieved = sum(alg_bytes) / (ms * 1e-3) / 1e9
    else:
        achieved = sum(alg_bytes) / (sum(mean_stage) * 1e-3) / 1e9  # GB/s over the stage kernels
    return dict(
        precision=precision, value=dof * 3 / (ms * 1e-3), ms_per_step=ms, err_vs_oracle=err,
        err_bound=ERR_BOUND[precision], dof=dof, launches=launches, steady_ms=steady_ms,
        stage_us=[float(v * 1e3) for v in mean_stage], achieved_gbs=achieved,
        alg_bytes_per_step=sum(alg_bytes), e2e_value=dof * 3 / e2e_s, e2e_ms=e2e_s * 1e3,
        h2d=dof * 8, d2h=dof * 8, variant=variant, tile=tile,
    )


def measure_extra(torch, frsg, wl, precision, steps, warmup, stream, flush, integrator="ssp3"):
    """Throughput of another workload (FP64 or FP32 form): per-step events with the L2
    flush between steps, dt from the CFL condition refreshed every 20 steps outside the timed
    events, plus the stage-kernel duration (limiter launches, if any, timed with their
    stage).  integrator "rk4" times classical RK4 steps (four stages; per-stage time = step
    time / 4)."""
    rk4 = integrator == "rk4"
    nst = 4 if rk4 else 3
    lim = bool(wl["solver"].get("limiter"))
    E, Np, M, S = workload_sizes(wl)
    dof = E * Np * M * S
    esz = 8 if precision == "fp64" else 4
    s = frsg.Solver(stream=stream.cuda_stream, precision=precision, **wl["solver"])
    s.autotune()
    nodes = s.nodes()
    if "boundary" in wl:
        for side, fn in wl["boundary"].items():
            s.set_boundary_nodal(side, workloads.boundary_values(fn, nodes[-1]))
    if len(nodes) == 2:
        s.set_initial_nodal(workloads.nodal_values(wl["ic"], nodes[0], nodes[1]))
    else:
        s.set_initial_nodal(workloads.nodal_values(wl["ic"], nodes[0], nodes[2], nodes[1]))
    # half the CFL number of the correctness runs, refreshed every 20 steps outside the timed
    # events: the Euler wave speeds grow after t = 0.  With the limiter on, the state is
    # limited before each refresh (a projection discontinuous in z, or a filtered stage
    # output, can leave inadmissible z-node states that the next stage would limit anyway).
    cfl = 0.5 * wl["cfl"]

    def refresh_dt():
        if lim:
            s.limit()
        return s.cfl_dt(cfl)
    dt = refresh_dt()
    advance = s.rk4_step if rk4 else s.rk_step
    with torch.cuda.stream(stream):
        advance(dt, warmup, graph=True)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for i in range(steps):
            if i % 20 == 0:
                dt = refresh_dt()
            flush.zero_()
            starts[i].record(stream)
            advance(dt, 1, graph=True)
            ends[i].record(stream)
        stream.synchronize()
        step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        kst = 0 if rk4 else min(steps, 50)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(kst)]
        for i in range(kst):
            flush.zero_()
            evs[i][0].record(stream)
            for st in range(3):
                s.stage(st, dt)
                evs[i][st + 1].record(stream)
        stream.synchronize()
    s.check()
    s.close()
    ms = float(np.mean(step_ms))
    if rk4:
        stage = np.full(4, ms / 4)
        alg = (3 + 5 + 5 + 3) * esz * dof      # arrays per stage: y, u, sum of residuals
    else:
        stage = np.mean(np.array([[evs[i][k].elapsed_time(evs[i][k + 1]) for k in range(3)]
                                  for i in range(kst)]), axis=0)
        alg = (2 + 3 + 3) * esz * dof
    return dict(value=dof * nst / (ms * 1e-3), ms_per_step=ms, dof=dof, stage_us=[float(v * 1e3) for v in stage],
                achieved_gbs=alg / (float(np.sum(stage)) * 1e-3) / 1e9, limiter=lim, integrator=integrator,
                filter=wl["solver"].get("filter"), flux=wl["solver"].get("flux", "llf"))


def measure_batch(torch, frsg, precision, steps, warmup, stream, flush):
    """The batched workload: 256 seeded Burgers problems of uneven size and order, advanced
    together by one persistent launch per stage (graph-replayed), L2 flushed between steps."""
    wls = workloads.burgers_batch()
    solvers = []
    dof = 0
    for wl in wls:
        sv = frsg.Solver(stream=stream.cuda_stream, precision=precision, **wl["solver"])
        x, z = sv.nodes()
        sv.set_initial_nodal(workloads.nodal_values(wl["ic"], x, z))
        solvers.append(sv)
        E, Np, M, S = workload_sizes(wl)
        dof += E * Np * M * S
    dts = np.array([wl["cfl"] * (wl["solver"]["x1"] - wl["solver"]["x0"]) / wl["solver"]["nx"] / wl["lam0"]
                    for wl in wls])
    b = frsg.Batch(solvers, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        b.rk_step(dts, warmup)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        l0 = b.launch_count()
        for i in range(steps):
            flush.zero_()
            starts[i].record(stream)
            b.rk_step(dts, 1)
            ends[i].record(stream)
        stream.synchronize()
    launches = b.launch_count() - l0
    for sv in solvers:
        sv.check()
    ms = float(np.mean([a.elapsed_time(c) for a, c in zip(starts, ends)]))
    info = b.info()
    b.close()
    for sv in solvers:
        sv.close()
    esz = 8 if precision == "fp64" else 4
    alg = (2 + 3 + 3) * esz * dof
    return dict(value=dof * 3 / (ms * 1e-3), ms_per_step=ms, dof=dof, members=len(wls), launches_per_step=launches / steps,
                step_gbs=alg / (ms * 1e-3) / 1e9, **info)


def measure_adjoint(torch, frsg, stream, nsteps=64, k=16):
    """Time of fr_sg_adjoint over the time of fr_sg_forward_record for the same run
    (Burgers, 1024 elements, FP64, checkpoints every k steps)."""
    wl = workloads.burgers_1d()
    sv = frsg.Solver(stream=stream.cuda_stream, **wl["solver"])
    x, z = sv.nodes()
    sv.set_initial_nodal(workloads.nodal_values(wl["ic"], x, z))
    u0 = torch.empty(sv.state_shape, dtype=torch.float64, device="cuda")
    sv.get_state(u0)
    dt = wl["cfl"] * (wl["solver"]["x1"] - wl["solver"]["x0"]) / wl["solver"]["nx"] / wl["lam0"]
    lam = torch.zeros_like(u0)
    g = torch.empty_like(u0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fw, bw = [], []
    with torch.cuda.stream(stream):
        for rep in range(4):
            sv.set_state(u0)
            sv.forward_record(dt, nsteps, k)
            lam.zero_()
            lam[:, :, 0, 0] = 1.0
            stream.synchronize()
            ev[0].record(stream)
            sv.forward_record(dt, nsteps, k)
            ev[1].record(stream)
            sv.adjoint(lam, g)
            ev[2].record(stream)
            stream.synchronize()
            if rep > 0:
                fw.append(ev[0].elapsed_time(ev[1]))
                bw.append(ev[1].elapsed_time(ev[2]))
    sv.check()
    sv.close()
    f, a = float(np.median(fw)), float(np.median(bw))
    return dict(workload=wl["name"], steps=nsteps, checkpoint_every=k, forward_ms=f, adjoint_ms=a, ratio=a / f)


def cpu_baseline(wl, seconds):
    import oracle
    from oracle import integrate, tables
    kw = dict(wl["solver"])
    prob = oracle.Problem(**kw)
    tabs = prob.tabs()
    u = integrate.project_initial(prob, wl["ic"])
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    E, Np, M, S = workload_sizes(wl)
    dof = E * Np * M * S
    n = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds or n < 2:
        u = integrate.ssp_rk3_step(prob, tabs, u, dt)
        n += 1
    t = time.perf_counter() - t0
    del tables
    return dict(value=dof * 3 * n / t, unit=UNIT, cores=1, kind="oracle",
                sample=f"{n} SSP-RK3 steps of the full {wl['name']} workload from t=0 "
                       f"(numpy FP64 oracle, single thread), {t:.1f} s")


def oracle_reference(wl, nsteps):
    import oracle
    from oracle import integrate
    prob = oracle.Problem(**wl["solver"])
    u = integrate.project_initial(prob, wl["ic"])
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    return integrate.run(prob, u, dt, nsteps)


def run_only(args):
    """One extra measurement alone, both forms where they apply (profiling aid)."""
    import torch
    from paper_2112_05946_gb300 import build as _b
    from paper_2112_05946_gb300 import frsg
    _b.build()
    frsg.load_library()
    tune_file = load_tune_cache(frsg)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if args.only == "burgers":
        wl = workloads.burgers_1d()
        ref = oracle_reference(wl, ACC_STEPS)
        out = measure_form(torch, frsg, wl, "fp32", args.steps, args.warmup, stream, flush, ref)
    elif args.only == "batch":
        out = {p: measure_batch(torch, frsg, p, args.steps, args.warmup, stream, flush) for p in ("fp64", "fp32")}
    elif args.only == "adjoint":
        out = measure_adjoint(torch, frsg, stream)
    else:
        wl = workloads.ALL[args.only]()
        out = {p: measure_extra(torch, frsg, wl, p, args.steps, args.warmup, stream, flush) for p in ("fp64", "fp32")}
    print(json.dumps({"only": args.only, "result": out}))
    if tune_file:
        frsg.tune_cache_save(tune_file)


def run_ours(args):
    import torch
    if args.only:
        return run_only(args)
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2112_05946_gb300 import build as _b
    from paper_2112_05946_gb300 import frsg
    if rank == 0 or not os.path.exists(frsg.LIB_PATH):
        _b.build()
    if world > 1:
        torch.distributed.barrier()
    frsg.load_library()
    tune_file = load_tune_cache(frsg)
    wl = workloads.ALL[args.workload]()
    ref = oracle_reference(wl, ACC_STEPS)
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    sampler = ClockSampler(local)
    sampler.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    forms = {}
    for prec in ("fp64", "fp32"):
        forms[prec] = measure_form(torch, frsg, wl, prec, args.steps, args.warmup, stream, flush, ref)
    extra = {}
    batch = {}
    adj = None
    if not args.no_extra:
        bsteps = max(3, min(args.steps, 50))
        batch = {prec: measure_batch(torch, frsg, prec, bsteps, 3, stream, flush) for prec in ("fp64", "fp32")}
        adj = measure_adjoint(torch, frsg, stream)
        xsteps = max(3, min(args.steps, 100))
        for name in ("sod", "shock_vortex"):
            ewl = workloads.ALL[name]()
            extra[ewl["name"]] = {prec: measure_extra(torch, frsg, ewl, prec, xsteps, 3, stream, flush)
                                  for prec in ("fp64", "fp32")}
        # the headline workload with the Lasso filter (every element), and with classical RK4
        lwl = workloads.burgers_1d()
        lwl["solver"].update(filter="lasso", sensor=False)
        extra[lwl["name"] + "_lasso"] = {prec: measure_extra(torch, frsg, lwl, prec, xsteps, 3, stream, flush)
                                         for prec in ("fp64", "fp32")}
        rwl = workloads.burgers_1d()
        extra[rwl["name"] + "_rk4"] = {prec: measure_extra(torch, frsg, rwl, prec, xsteps, 3, stream, flush, "rk4")
                                       for prec in ("fp64", "fp32")}
        # the paper's second Sod case (stochastic shock location, HLL, Lasso) at 4096 elements
        hwl = workloads.sod_location_1d(nx=4096)
        extra[hwl["name"]] = {prec: measure_extra(torch, frsg, hwl, prec, xsteps, 3, stream, flush)
                              for prec in ("fp64", "fp32")}
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()

    ok = [f for f in forms.values() if f["err_vs_oracle"] <= f["err_bound"]]
    chosen = max(ok, key=lambda f: f["value"]) if ok else forms["fp64"]
    ms = max_over_ranks(torch, chosen["ms_per_step"], world, "cuda")
    value = whole_job_value(world, chosen["dof"], 3, ms)

    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        with open(pk) as f:
            peaks = json.load(f)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    kname = {0: "stage1d_kernel", 1: "stage1d_wide_kernel", 2: "stage1d_step_kernel",
             3: "step1d_fused_kernel"}[chosen["variant"]]
    # DRAM bytes of one launch from the ncu capture of this kernel build; null for a layout
    # without a capture of the current build
    traffic = MEASURED_TRAFFIC.get((kname, chosen["precision"], chosen["tile"]))
    roofline = {"bound": "hbm", "achieved": round(chosen["achieved_gbs"], 2), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(chosen["achieved_gbs"] / hbm_peak, 5), "traffic": traffic,
                "kernel": kname, "peak_source": "measured" if peaks else "fallback",
                "alg_bytes_per_step": chosen["alg_bytes_per_step"]}
    if chosen["variant"] in (2, 3):
        # one launch per step: the timed launch is the step (fr_sg_stage runs single stages in
        # another layout, so its times do not describe this kernel)
        roofline["launch_us"] = round(chosen["ms_per_step"] * 1e3, 3)
    else:
        roofline["stage_us"] = chosen["stage_us"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_seconds)

    E, Np, M, S = workload_sizes(wl)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if chosen["precision"] == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "elements": E, "P": wl["solver"]["P"], "N": wl["solver"]["N"],
                   "Q": wl["solver"]["Q"], "S": S, "dof": E * Np * M * S, "filter": "exp+detector",
                   "l2": "256 MiB memset between timed steps (state 0.3 MB < L2)",
                   "parallelism": f"replicas x{world}"},
        "chosen": chosen["precision"],
        "forms": {k: {"value": v["value"], "ms_per_step": v["ms_per_step"], "rel_l2_vs_oracle": v["err_vs_oracle"],
                      "err_bound": v["err_bound"], "steady_ms_per_step": v["steady_ms"],
                      "stage_us": v["stage_us"], "variant": v["variant"], "tile": v["tile"]}
                  for k, v in forms.items()},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": chosen["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": chosen["h2d"],
                "d2h_bytes_per_step": chosen["d2h"], "ms_per_step": chosen["e2e_ms"]},
        "gpu_launches": chosen["launches"],
        "clocks": clocks,
        "batched": {"workload": "burgers_batch0: 256 problems, E 64-2048, P 1-4, N 2-10, Q 2N",
                    **{p: {k2: (float(v2) if isinstance(v2, (int, float)) else v2) for k2, v2 in f.items()}
                       for p, f in batch.items()}},
        "adjoint": adj,
        "other_workloads": {
            k: {p: {"value": f["value"], "ms_per_step": f["ms_per_step"], "dof": f["dof"], "stage_us": f["stage_us"],
                    "stage_gbs": f["achieved_gbs"], "stage_hbm_frac": f["achieved_gbs"] / hbm_peak,
                    "limiter": f["limiter"], "integrator": f["integrator"], "filter": f["filter"],
                    "flux": f["flux"]}
                for p, f in v.items()}
            for k, v in extra.items()},
    }
    if rank == 0:
        print(json.dumps(line))
        if tune_file:
            frsg.tune_cache_save(tune_file)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from oracle import integrate
    wl = workloads.ALL[args.workload]()
    prob = oracle.Problem(**wl["solver"])
    tabs = prob.tabs()
    u = integrate.project_initial(prob, wl["ic"])
    dt = wl["cfl"] * prob.dx / wl["lam0"]
    E, Np, M, S = workload_sizes(wl)
    dof = E * Np * M * S
    for _ in range(args.warmup):
        u = integrate.ssp_rk3_step(prob, tabs, u, dt)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = integrate.ssp_rk3_step(prob, tabs, u, dt)
    t = time.perf_counter() - t0
    value = dof * 3 * args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["name"], "elements": E, "P": wl["solver"]["P"], "N": wl["solver"]["N"],
                   "Q": wl["solver"]["Q"], "S": S, "dof": dof},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} timed SSP-RK3 steps of the full {wl['name']} workload "
                                   f"after {args.warmup} warm-up steps (numpy FP64 oracle, single thread)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
