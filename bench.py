#!/usr/bin/env python3
"""Benchmark of the FourierSMT hot path on B300: fwd+adjoint xBDD nodes/s.

A step is one annealing stage of Alg. 2 over one batch of restarts: `iters`
iterations of [relax -> forward COP -> adjoint -> PGD + projection -> ||g||^2
test], then round + exact check + ERWA.  The stage runs from a captured CUDA
graph (fused form).  value = decision-node visits of the forward+adjoint sweep
(nodes in C_sigma x restarts x iterations run) per second, whole job.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload large_scheduling] [--iters 20] [--tts SECONDS]

Under torchrun (N > 1) every rank runs an independent replica (its own restart
seeds; the paper runs 8 independent replicas): weak scaling, no collective on
the data path; rank 0 prints the max-over-ranks time.  In the time-to-SAT runs
the replicas share one [SAT verified, out of time] flag per stage.

Other modes: --workload (any entry of WORKLOADS), --gradient-time (the paper's
gradient-time experiment on the random hybrid benchmark), --no-tts-plain (skip
the plain form's time to SAT, one seed by default), --impl reference (the FP64
oracle on the host).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import instances as W  # noqa: E402

METRIC = "fwd+adjoint xBDD nodes/s"
UNIT = "nodes/s"

WORKLOADS = {
    "random_hybrid": (lambda: W.random_hybrid(1006, 1000), 100),
    "large_scheduling": (lambda: W.large_scheduling(1005), 512),
    "large_scheduling_400": (lambda: W.large_scheduling(1005, n_jobs=400), 512),
    # the encoding read literally: 1,000 jobs on 20 workers (5 index bits, 6,000 variables)
    "large_scheduling_lit": (lambda: W.large_scheduling(1005, n_workers=20, n_jobs=1000, n_late=6), 512),
    "placement2d": (lambda: W.placement2d(1003), 1024),
    # the same rectangles with the paper's style of non-overlap: a plain 4-atom OR, no selectors
    "placement2d_nosel": (lambda: W.placement2d(1003, selectors=False), 1024),
    # the paper's 3D placement encoding: 64 macros x 8 layers, 896 modules
    "placement3d": (lambda: W.placement3d(1007), 512),
    "jobshop": (lambda: W.jobshop(1002), 256),
    "uneven_batch": (lambda: W.concat(W.uneven_batch(1004), "uneven_batch"), 32),
    "tiny_random": (lambda: W.tiny_random(1001), 64),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="large_scheduling", choices=list(WORKLOADS))
    p.add_argument("--iters", type=int, default=20, help="PGD iterations per stage (step)")
    p.add_argument("--eta", type=float, default=None)
    p.add_argument("--tts", type=float, default=150.0,
                   help="time-to-SAT budget in seconds per form (0 = skip)")
    p.add_argument("--no-tts-plain", dest="tts_plain", action="store_false",
                   help="skip the time-to-SAT run of the plain (unfused) form")
    p.add_argument("--tts-plain-seeds", type=int, default=1,
                   help="initial-point seeds of the plain form's time-to-SAT (the first ones of the fused form's)")
    p.add_argument("--tts-eta", type=float, default=0.2)
    p.add_argument("--tts-iters", type=int, default=20, help="PGD iterations per stage in the time-to-SAT runs")
    p.add_argument("--tts-trace", default=None,
                   help="JSON-lines file for the per-stage records of the time-to-SAT runs (Solver.anneal log)")
    p.add_argument("--tts-seeds", type=int, default=5,
                   help="initial-point seeds per form; the median is PAR-2 (a miss counts twice the limit)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--roofline-launches", type=int, default=10)
    p.add_argument("--gradient-time", action="store_true",
                   help="the paper's gradient-time experiment on the random hybrid benchmark instead of the bench")
    p.add_argument("--gt-instances", type=int, default=10, help="instances per n in --gradient-time")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(rank):
    """Restart seed of a replica: every rank draws its own initial points."""
    return 7 + 1000 * rank


def max_over_ranks(x, device="cpu"):
    """Max of a number over the ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def per_instance_plain(args, R, eta):
    """The uneven batch's members as separate instances: one compiled object and one
    plain-form solver per member (same R, eta, iterations and sigma schedule as the
    batched run), one stage of every member per step, timed with CUDA events."""
    import torch
    from paper_2603_22877_b300 import Solver
    from paper_2603_22877_b300.engine import Problem
    members = []
    for k, inst in enumerate(W.uneven_batch(1004)):
        P = Problem.from_instance(inst)
        comp = P.compile().upload()
        S = Solver(P, comp, R, eta=eta, b_scale=inst.scale, t_max=args.iters, sweeps=20, use_graph=False,
                   form="plain")
        a0, b0 = W.initial_point(inst, R, seed=replica_seed(0) + k)
        S.reset(a0, b0)
        members.append((S, [inst.scale / (0.1 * t) for t in range(1, 21)]))

    def step(k):
        for S, sched in members:
            S.stage(sched[k % len(sched)], k + 1)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        step(args.warmup + k)
    e1.record()
    torch.cuda.synchronize()
    return {"instances": len(members), "ms_per_step": e0.elapsed_time(e1) / args.steps,
            "form": "plain, one solver per instance, no graph"}


def kernel_name(launch):
    """The forward + adjoint kernel that a launch configuration runs, as the launch list names it."""
    rpl = launch["restarts_per_lane"]
    return {"warp": "k_fused<1> (one warp per constraint, forward + adjoint)",
            "chunked": f"k_chunked<1, {rpl}> (chunked, ahead-of-time generic diagram pass)",
            "jit": f"fsmt_jit_adj_{rpl} (chunked, run-time generated routines and the generic pass)",
            "wide": f"fsmt_jit_wide_adj_{rpl} (chunked, run-time generated routines for every shape)",
            }.get(launch["variant"], str(launch["variant"]))


def whole_job_rate(units_per_rank, ws, ms):
    """Units of all ranks per second over the slowest rank's time (weak scaling)."""
    return units_per_rank * ws / (ms / 1000.0)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


# ---------------------------------------------------------------------------- ncu traffic record
KERNEL_SOURCES = ["paper_2603_22877_b300/csrc/fsmt_chunked.cuh", "paper_2603_22877_b300/csrc/fsmt_devview.cuh",
                  "paper_2603_22877_b300/csrc/fsmt_jit.cpp"]


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(workload, R):
    """DRAM bytes per launch of the fused kernel from the committed ncu summary,
    or None when the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"fsmt_jit_wide_adj.{workload}.R{R}.md")
    if not os.path.exists(path):
        return None, "no ncu summary for this workload"
    rec = {}
    with open(path) as f:
        for line in f:
            if line.startswith("- ") and ": " in line:
                k, v = line[2:].strip().split(": ", 1)
                rec[k.strip("`")] = v.strip().strip("`")
    if rec.get("kernel_sources_sha256") != kernel_sources_sha256():
        return None, f"{os.path.relpath(path, ROOT)} predates the current kernel sources"
    return float(rec["traffic_bytes_per_launch"]), os.path.relpath(path, ROOT)


# ---------------------------------------------------------------------------- oracle timing
def oracle_sample_rate(inst, R, a, b, w, sigma, budget_s):
    """The FP64 oracle (as it stands) over a bounded prefix of the constraints of C_sigma.

    Returns (nodes/s, constraints sampled, node-restart visits, seconds)."""
    from oracle import objective as OBJ
    D = OBJ.Diagrams(inst)
    a64, b64, w64 = a.astype(np.float64), b.astype(np.float64), w.astype(np.float64)
    oc = OBJ.objective_constraints(inst)
    t0 = time.perf_counter()
    visits, k = 0, 0
    while k < len(oc) and time.perf_counter() - t0 < budget_s:
        c = oc[k]
        OBJ.constraint_contrib(inst, D, c, a64, b64, w64[c], sigma)
        visits += len(D[c][0]) * R
        k += 1
    dt = time.perf_counter() - t0
    return visits / dt, k, visits, dt


def reference_arm(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    make, R = WORKLOADS[args.workload]
    inst = make()
    a, b = W.initial_point(inst, R, seed=7)
    w = np.ones((inst.n_cons, R), np.float32)
    sigma = inst.scale / (0.1 * 10)
    budget = 3.0
    for _ in range(args.warmup):
        oracle_sample_rate(inst, R, a, b, w, sigma, budget)
    visits, secs, ks = 0, 0.0, []
    for _ in range(args.steps):
        _, k, v, dt = oracle_sample_rate(inst, R, a, b, w, sigma, budget)
        visits += v
        secs += dt
        ks.append(k)
    value = visits / secs
    sample = (f"first {max(ks)} constraints of C_sigma x {R} restarts per step (~{budget:.0f} s of FP64 numpy "
              f"forward+adjoint each), {inst.name}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": inst.name, "restarts": R, "n_vars": inst.n_bool + inst.n_real,
                       "n_cons": inst.n_cons},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- our arm
def our_arm(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    from paper_2603_22877_b300 import Solver, build
    from paper_2603_22877_b300.engine import Problem
    build.build()
    make, R = WORKLOADS[args.workload]
    inst = make()
    t_c = time.perf_counter()
    P = Problem.from_instance(inst)
    comp = P.compile()
    compile_s = time.perf_counter() - t_c
    t_c = time.perf_counter()
    comp.upload()                       # device copy + run-time generated routines
    torch.cuda.synchronize()
    upload_s = time.perf_counter() - t_c
    info = comp.info
    eta = args.eta if args.eta is not None else 0.02
    a0, b0 = W.initial_point(inst, R, seed=replica_seed(rank))
    S = Solver(P, comp, R, eta=eta, b_scale=inst.scale, t_max=args.iters, sweeps=20, use_graph=True)
    S.reset(a0, b0)
    sched = [inst.scale / (0.1 * t) for t in range(1, 21)]
    launch = S.tune(sched[0]).as_dict()  # autotuned kernel configuration (fsmt_autotune)
    stream = torch.cuda.current_stream()
    nodes = info["n_obj_nodes"]

    def step(k):
        S.stage(sched[k % len(sched)], k + 1)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        step(args.warmup + k)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # a stage stops early only when every restart has converged: count what ran
    iters_per_step = int(S.iters.max().item())
    ms = max_over_ranks(ms, dev)
    clk = clocks.stop()
    value = whole_job_rate(nodes * R * iters_per_step * args.steps, ws, ms)

    # end to end through the C ABI with host buffers (copies inside the timed region)
    a_h = torch.from_numpy(a0).pin_memory()
    b_h = torch.from_numpy(b0).pin_memory()
    nu_h = torch.zeros(R, dtype=torch.int32).pin_memory()
    ob_h = torch.zeros(R, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        S.stage_host(sched[k % len(sched)], k + 1, a_h.numpy(), b_h.numpy(), nu_h.numpy(), ob_h.numpy())
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev)
    e2e_value = whole_job_rate(nodes * R * iters_per_step * args.steps, ws, 1000.0 * e2e_s)
    h2d = (inst.n_bool + inst.n_real) * R * 4
    d2h = R * 8

    # roofline of the dominant kernel: the fused forward+adjoint, timed alone with events
    da, db, dw = S.a, S.b, S.w
    ga, gb = torch.zeros_like(da), torch.zeros_like(db)
    obj = torch.zeros(R, device=dev)
    sigma = sched[9]
    for _ in range(2):
        comp.adjoint(R, sigma, dw, da, db, ga, gb, obj=obj)
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.roofline_launches):
        comp.adjoint(R, sigma, dw, da, db, ga, gb, obj=obj)
    f1.record(stream)
    torch.cuda.synchronize()
    fused_ms = f0.elapsed_time(f1) / args.roofline_launches  # includes the three small memsets
    peaks, peak_kind = load_peaks()
    # The fused kernel is bound by instruction issue, not by DRAM: its DRAM
    # traffic is the algorithmic minimum (structure once, w and the state once)
    # and runs at a few percent of HBM bandwidth.  Its roofline is FP32 ALU:
    # 10 flops per decision-node visit (Alg. 3: two FMA; Alg. 4: one subtract,
    # one FMA; adjoint: one FMA, counted as in DESIGN) against 148 SMs x 128 FP32
    # lanes x 2 flops x the maximum SM clock.
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    alu_peak = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12
    alg_flops = 10.0 * nodes * R
    structure = nodes * 8 + info["n_atoms"] * 17 + info["atom_nnz"] * 8 + info["n_obj_cons"] * 9
    state = 4 * R * (info["n_obj_cons"] + 2 * (inst.n_bool + inst.n_real) + 1)
    alg_bytes = structure + state
    achieved = alg_flops / (fused_ms / 1000.0) / 1e12
    traffic, traffic_note = profiled_traffic(args.workload, R)
    roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                "frac": achieved / alu_peak, "traffic": traffic,
                "peak_kind": f"derived: 148 SMs x 128 FP32 lanes x 2 flops (FMA) x {sm_mhz:.0f} MHz",
                "kernel": kernel_name(launch),
                "kernel_ms": fused_ms, "algorithmic_flops": alg_flops, "traffic_source": traffic_note,
                "node_visits_per_s": nodes * R / (fused_ms / 1000.0),
                "hbm": {"algorithmic_bytes": alg_bytes, "achieved_gbs": alg_bytes / (fused_ms / 1000.0) / 1e9,
                        "peak_gbs": peaks["hbm_gbs"], "frac": alg_bytes / (fused_ms / 1000.0) / 1e9 / peaks["hbm_gbs"],
                        "peak_kind": peak_kind}}

    # plain (unfused) form of the same forward+adjoint, for comparison
    plain = None
    try:
        nwork = comp.plain_work(R)
        if nwork * 4 < 0.6 * torch.cuda.mem_get_info()[0]:
            work = torch.empty(nwork, device=dev)
            for _ in range(2):
                comp.forward_plain(R, sigma, dw, da, db, work, obj=obj)
                comp.adjoint_plain(R, sigma, dw, da, db, work, ga, gb)
            torch.cuda.synchronize()
            f0.record(stream)
            for _ in range(3):
                comp.forward_plain(R, sigma, dw, da, db, work, obj=obj)
                comp.adjoint_plain(R, sigma, dw, da, db, work, ga, gb)
            f1.record(stream)
            torch.cuda.synchronize()
            pms = f0.elapsed_time(f1) / 3
            plain = {"ms_per_fwd_adj": pms, "node_visits_per_s": nodes * R / (pms / 1000.0),
                     "fused_speedup": pms / fused_ms}
            del work
    except Exception as e:  # report, never hide
        plain = {"error": str(e)}

    # the uneven batch member by member: each instance its own compiled object and a
    # plain stage per step (forward, adjoint and PGD launched from Python, no graph) --
    # the per-instance form that the one batched fused launch per stage replaces
    per_instance = None
    if args.workload == "uneven_batch":
        try:
            per_instance = per_instance_plain(args, R, eta)
            per_instance["batched_speedup"] = per_instance["ms_per_step"] / (ms / args.steps)
        except Exception as e:  # report, never hide
            per_instance = {"error": str(e)}

    # time to the first exactly verified SAT: Alg. 2 from the same initial points,
    # the schedule 1/sigma = 0.1, 0.2, ... in units of the instance scale,
    # continued past 2.0 until SAT or the time limit
    # (one run per initial-point seed, each from a fresh solver, graph capture included;
    # the first seed's points are the bench's own).  Under torchrun every rank is a
    # replica with its own seeds; they share a [SAT verified, out of time] flag per stage
    # and all stop at the first stage where some replica verified SAT.
    tts = None
    share = None
    if ws > 1:
        from paper_2603_22877_b300 import max_over_replicas
        share = max_over_replicas("cuda" if torch.distributed.get_backend() == "nccl" else "cpu")
    if args.tts > 0:
        tts = {"eta": args.tts_eta, "iters_per_stage": args.tts_iters, "limit_s": args.tts}
        sched_tts = [inst.scale / (0.1 * t) for t in range(1, 1001)]
        for form in ("fused", "plain") if args.tts_plain else ("fused",):
            runs = []
            for s in range(max(1, args.tts_seeds if form == "fused" else min(args.tts_plain_seeds, args.tts_seeds))):
                pa, pb = (a0, b0) if s == 0 else W.initial_point(inst, R, seed=replica_seed(rank) + 100000 * s)
                S2 = Solver(P, comp, R, eta=args.tts_eta, b_scale=inst.scale, t_max=args.tts_iters, sweeps=20,
                            use_graph=True, form=form)
                S2.reset(pa, pb)
                torch.cuda.synchronize()
                log = None
                if args.tts_trace and rank == 0:
                    from paper_2603_22877_b300 import jsonl_log
                    log = jsonl_log(args.tts_trace)
                    log({"form": form, "seed": s, "workload": args.workload, "restarts": R})
                res = S2.anneal(sched_tts, time_limit=args.tts, share=share, log=log)
                if log is not None:
                    log.close()
                solved = res["sat"] or res["stopped_by_peer"]   # by this replica or another
                rec = {"sat": solved, "seconds": res["seconds"], "stage": res["stages_run"] if solved else None,
                       "restart": res["restart"], "stages_run": res["stages_run"], "best_unsat": res["best_unsat"]}
                if ws > 1:
                    rec["found_here"] = res["sat"]
                if solved:
                    rec["inv_sigma_over_scale"] = round(0.1 * res["stages_run"], 1)
                runs.append(rec)
                del S2
                torch.cuda.empty_cache()
            par2 = [r["seconds"] if r["sat"] else 2 * args.tts for r in runs]
            tts[form] = {"median_s_par2": float(np.median(par2)), "solved": sum(r["sat"] for r in runs),
                         "seeds": len(runs), "runs": runs}
        if "plain" in tts and tts["fused"]["runs"][0]["sat"] and tts["plain"]["runs"][0]["sat"]:
            # same initial points, same schedule: the batched fused form against the plain one
            tts["plain_over_fused_seed0"] = tts["plain"]["runs"][0]["seconds"] / tts["fused"]["runs"][0]["seconds"]

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:  # the host baseline runs at N = 1 only
        rate, k, v, dt = oracle_sample_rate(inst, R, a0, b0, np.ones((inst.n_cons, R), np.float32), sigma, 15.0)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {k} constraints of C_sigma x {R} restarts, FP64 numpy forward+adjoint, "
                         f"{dt:.1f} s on the host"}
    # per stage: parameters, stage start, weight sums; per iteration: iteration
    # start, fused forward+adjoint, one PGD kernel per variable class, convergence
    # test; then round + check: over the chunks for C_sigma, one warp per constraint
    # for the rest (graph iterations past convergence still launch)
    checks = (info["n_chunks"] > 0) + (info["n_chunks"] == 0 or inst.n_cons > info["n_obj_cons"])
    launches_per_step = 3 + args.iters * (3 + (inst.n_bool > 0) + (info["n_free_reals"] > 0) +
                                          (info["n_components"] > 0)) + checks
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "restarts": R, "n_vars": inst.n_bool + inst.n_real,
                           "n_bool": inst.n_bool, "n_real": inst.n_real, "n_cons": inst.n_cons,
                           "n_obj_cons": info["n_obj_cons"], "n_obj_nodes": nodes, "atoms": inst.n_atoms,
                           "iters_per_step": iters_per_step, "eta": eta, "form": "fused + CUDA graph",
                           "l2": "inputs larger than L2 (diagrams + weights > 126 MB)",
                           "compile_s": compile_s, "upload_s": upload_s, "parallelism": f"replicas x{ws}",
                           "launch": launch},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches_per_step * args.steps, "clocks": clk, "plain": plain,
                "per_instance": per_instance,
                "time_to_sat": tts}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# Per-instance average gradient time of the paper's own solver on the random
# hybrid benchmark, averaged over the 10 instances of each n: (CPU, dual EPYC 9654
# at 64 threads; GPU, one L40S), ms (Suppl. Note "Gradient Computation Time",
# Table gradient-time).  Context from other hardware, not a target of this line.
PAPER_GRADIENT_MS = {100: (4.98, 12.70), 200: (21.78, 13.64), 300: (34.15, 12.77), 400: (43.14, 12.80),
                     500: (48.40, 12.60), 600: (56.27, 12.79), 700: (62.40, 12.76), 800: (69.08, 12.84),
                     900: (77.37, 12.87), 1000: (84.35, 12.65)}


def gradient_time(args):
    """The gradient-time experiment (Suppl. Note "Gradient Computation Time") on
    the random hybrid benchmark: per instance, gradients at 10,000 random points in
    100 groups of 100 points, one sigma per group with 1/sigma = 0.00, 0.01, ...,
    0.99 (in units of the reals' [0, 1] range).  One group is one batched forward +
    adjoint call at R = 100 (fused kernel when one fits the instance, else the plain
    form); the 100 calls of an instance are timed together with CUDA events.  The
    oracle (FP64 numpy, one core) is timed on one group per n."""
    import torch
    from paper_2603_22877_b300 import build
    from paper_2603_22877_b300.engine import Problem
    build.build()
    R, groups = 100, 100
    inv = [0.01 * g for g in range(groups)]
    sig = [math.inf if x == 0 else 1.0 / x for x in inv]
    per_n = {}
    for n in range(100, 1001, 100):
        times, forms = [], set()
        for k in range(args.gt_instances):
            inst = W.random_hybrid(1006 + 10 * k, n)
            comp = Problem.from_instance(inst).compile().upload()
            fused_ok = bool(comp.info["fused_ok"]) or comp.info["n_chunks"] > 0
            rng = np.random.default_rng(7 + k)
            a = torch.from_numpy(rng.uniform(-1, 1, (groups, n, R)).astype(np.float32)).cuda()
            b = torch.from_numpy(rng.uniform(0, 1, (groups, n, R)).astype(np.float32)).cuda()
            w = torch.ones((inst.n_cons, R), device="cuda")
            ga, gb = torch.zeros((n, R), device="cuda"), torch.zeros((n, R), device="cuda")
            obj = torch.zeros(R, device="cuda")
            work = torch.empty(comp.plain_work(R), device="cuda")
            if fused_ok:  # the autotuned fused configuration
                comp.autotune(R, sig[50], w, a[50], b[50], ga, gb, obj)

            def grad(g, fused):
                if fused:
                    comp.adjoint(R, sig[g], w, a[g], b[g], ga, gb, obj=obj)
                else:
                    comp.forward_plain(R, sig[g], w, a[g], b[g], work, obj=obj)
                    comp.adjoint_plain(R, sig[g], w, a[g], b[g], work, ga, gb)

            best = None
            for fused in ((True, False) if fused_ok else (False,)):  # the faster form counts
                for g in range(3):
                    grad(g, fused)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for g in range(groups):
                    grad(g, fused)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / groups
                if best is None or ms < best[0]:
                    best = (ms, "fused" if fused else "plain")
            times.append(best[0])
            forms.add(best[1])
            del work
            if k == 0:  # the oracle on one group of this n
                from oracle import objective as OBJ
                a64 = a[50].double().cpu().numpy()
                b64 = b[50].double().cpu().numpy()
                D = OBJ.Diagrams(inst)  # compiled once, outside the timed call
                t0 = time.perf_counter()
                OBJ.evaluate(inst, a64, b64, np.ones((inst.n_cons, R)), sig[50], diagrams=D)
                oracle_ms = 1000 * (time.perf_counter() - t0)
        gpu = float(np.mean(times))
        per_n[n] = {"gpu_ms_per_group": gpu, "gpu_us_per_point": 1000 * gpu / R, "form": "/".join(sorted(forms)),
                    "oracle_ms_per_group": oracle_ms, "instances": args.gt_instances,
                    "paper_cpu_ms": PAPER_GRADIENT_MS[n][0], "paper_gpu_ms": PAPER_GRADIENT_MS[n][1]}
        print(json.dumps({"n": n, **per_n[n]}), flush=True)
    line = {"metric": "gradient time (forward + adjoint of 100 points)", "unit": "ms", "higher_is_better": False,
            "data": "synthetic", "dtype": "f32", "config": {"workload": "random_hybrid", "points_per_group": R,
                                                            "groups": groups, "inv_sigma": "0.00..0.99"},
            "per_n": per_n}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.gradient_time:
        gradient_time(args)
        return
    if args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
