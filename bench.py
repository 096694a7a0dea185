#!/usr/bin/env python3
"""Benchmark of the FourierSMT hot path on B300: fwd+adjoint xBDD nodes/s.

A step is one annealing stage of Alg. 2 over one batch of restarts: `iters`
iterations of [relax -> forward COP -> adjoint -> PGD + projection -> ||g||^2
test], then round + exact check + ERWA.  The stage runs from a captured CUDA
graph, its iterations in the stage form the tuner found fastest (separate
launches, one persistent forward + adjoint + PGD kernel for the stage, or that
kernel once per iteration; all three timed in stage_forms_ms).  value =
decision-node visits of the forward+adjoint sweep (nodes in C_sigma x restarts x
iterations run) per second, whole job.

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
    p.add_argument("--tts-plain-seeds", type=int, default=5,
                   help="initial-point seeds of the plain form's time-to-SAT (the first ones of the fused form's)")
    p.add_argument("--tts-eta", type=float, default=0.2)
    p.add_argument("--tts-iters", type=int, default=20, help="PGD iterations per stage in the time-to-SAT runs")
    p.add_argument("--tts-trace", default=None,
                   help="JSON-lines file for the per-stage records of the time-to-SAT runs (Solver.anneal log)")
    p.add_argument("--tts-protocol", default="median", choices=["median", "first"],
                   help="under torchrun: 'median' runs every replica independently to its own SAT and reports "
                        "the median over replicas and seeds (the paper's protocol); 'first' stops all replicas "
                        "at the first stage where one of them verified SAT")
    p.add_argument("--tts-seeds", type=int, default=5,
                   help="initial-point seeds per form; the median is PAR-2 (a miss counts twice the limit)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--stage-form", default="auto", choices=["auto", "launches", "stage", "iteration"],
                   help="how a stage runs its PGD iterations: separate launches per iteration, one persistent "
                        "kernel for the stage, that kernel once per iteration, or auto (the fastest of the three, "
                        "timed by Solver.tune)")
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
def host_cpu():
    """(usable cores, CPU model) of this host."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return cores, model


def oracle_sample_rate(inst, R, a, b, sigma, budget_s, cons=None, cycle=False):
    """The FP64 oracle (as it stands, unit weights) over the constraints `cons` (default:
    C_sigma in id order), one after another until budget_s has passed, on this core
    (with cycle, starting again at the first when all are done).

    Returns (nodes/s, constraint evaluations, node-restart visits, seconds)."""
    from oracle import objective as OBJ
    D = OBJ.Diagrams(inst)
    a64, b64 = np.asarray(a, np.float64), np.asarray(b, np.float64)
    ones = np.ones(R)
    oc = OBJ.objective_constraints(inst) if cons is None else cons
    t0 = time.perf_counter()
    visits, k = 0, 0
    while (cycle or k < len(oc)) and oc and time.perf_counter() - t0 < budget_s:
        c = oc[k % len(oc)]
        OBJ.constraint_contrib(inst, D, c, a64, b64, ones, sigma)
        visits += len(D[c][0]) * R
        k += 1
    dt = time.perf_counter() - t0
    return visits / dt, k, visits, dt


def constraint_slice(inst, cons):
    """The instance restricted to the constraints `cons` and the atoms they name (atoms
    renumbered in order of first use; Booleans and reals unchanged), so that a worker
    process receives only its share of the input."""
    import dataclasses
    amap, ptr, var, coef, q0, rel = {}, [0], [], [], [], []
    kinds, params, cptr, lits = [], [], [0], []
    for c in cons:
        for l in inst.lits(c):
            vid = int(l) >> 1
            if vid >= inst.n_bool:
                i = vid - inst.n_bool
                if i not in amap:
                    amap[i] = len(amap)
                    v, cf, q, r = inst.atom(i)
                    var += list(v)
                    coef += list(cf)
                    ptr.append(len(var))
                    q0.append(q)
                    rel.append(r)
                vid = inst.n_bool + amap[i]
            lits.append(2 * vid + (int(l) & 1))
        kinds.append(int(inst.con_kind[c]))
        params.append(int(inst.con_param[c]))
        cptr.append(len(lits))
    return dataclasses.replace(
        inst, atom_ptr=np.asarray(ptr, np.int64), atom_var=np.asarray(var, np.int32),
        atom_coef=np.asarray(coef, np.int64), atom_q0=np.asarray(q0, np.int64), atom_rel=np.asarray(rel, np.int8),
        con_kind=np.asarray(kinds, np.int8), con_param=np.asarray(params, np.int32),
        con_ptr=np.asarray(cptr, np.int64), con_lits=np.asarray(lits, np.int32))


_W = {}


def _oracle_worker_init(shm_a, shape_a, shm_b, shape_b, R, sigma):
    from multiprocessing import shared_memory
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    sa = shared_memory.SharedMemory(name=shm_a) if shm_a else None
    sb = shared_memory.SharedMemory(name=shm_b) if shm_b else None
    _W.update(sa=sa, sb=sb, R=R, sigma=sigma,
              a=np.ndarray(shape_a, np.float64, buffer=sa.buf) if sa else np.zeros(shape_a),
              b=np.ndarray(shape_b, np.float64, buffer=sb.buf) if sb else np.zeros(shape_b))


def _oracle_worker(job):
    sub, start_at, budget_s = job
    while time.time() < start_at:   # every worker starts together
        time.sleep(0.001)
    _, k, v, dt = oracle_sample_rate(sub, _W["R"], _W["a"], _W["b"], _W["sigma"], budget_s,
                                     cons=list(range(sub.n_cons)), cycle=True)
    return v, dt, k


class OraclePool:
    """The FP64 oracle on `workers` processes at once (spawn context; the points shared
    through shared memory), each over its own block of `per_worker` consecutive
    constraints of C_sigma; run(budget) times one round of all of them together and
    returns (nodes/s = the sum of the workers' rates, constraints done, seconds)."""

    def __init__(self, inst, R, a, b, sigma, workers, per_worker):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        from oracle import objective as OBJ
        oc = OBJ.objective_constraints(inst)
        a64, b64 = np.ascontiguousarray(a, np.float64), np.ascontiguousarray(b, np.float64)
        self.shms, names = [], []
        for x in (a64, b64):
            if x.size:
                m = shared_memory.SharedMemory(create=True, size=x.nbytes)
                np.ndarray(x.shape, np.float64, buffer=m.buf)[...] = x
                self.shms.append(m)
                names.append(m.name)
            else:
                names.append(None)
        n = min(per_worker, len(oc))
        self.jobs = [constraint_slice(inst, [oc[(i * per_worker + j) % len(oc)] for j in range(n)])
                     for i in range(workers)]
        self.workers, self.per_worker = workers, per_worker
        self.pool = mp.get_context("spawn").Pool(workers, initializer=_oracle_worker_init,
                                                 initargs=(names[0], a64.shape, names[1], b64.shape, R, sigma))

    def run(self, budget_s):
        start_at = time.time() + 1.0 + 0.01 * self.workers
        res = self.pool.map(_oracle_worker, [(j, start_at, budget_s) for j in self.jobs], chunksize=1)
        return sum(v / dt for v, dt, _ in res), sum(k for _, _, k in res), max(dt for _, dt, _ in res)

    def close(self):
        self.pool.close()
        self.pool.join()
        for m in self.shms:
            m.close()
            m.unlink()


def cpu_baseline(inst, R, a, b, sigma, budget_s=10.0):
    """The FP64 oracle on this host: one core over C_sigma in order, then every usable
    core at once, each process over its own block of C_sigma (twice what one core got
    through in the same time); both in node visits per second."""
    cores, model = host_cpu()
    r1, k1, _, dt1 = oracle_sample_rate(inst, R, a, b, sigma, budget_s)
    per = max(64, 2 * k1)
    pool = OraclePool(inst, R, a, b, sigma, cores, per)
    try:
        rn, kn, dtn = pool.run(budget_s)
    finally:
        pool.close()
    return {"value": rn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"FP64 numpy forward+adjoint, {R} restarts: one core over the first {k1} constraints of "
                       f"C_sigma ({dt1:.1f} s); {cores} processes at once, each over its own block of {per} "
                       f"constraints of C_sigma ({dtn:.1f} s, {kn} constraints in all)"),
            "value_1core": r1, "value_allcores": rn, "cores_used": cores, "nproc": cores, "cpu_model": model}


def reference_arm(args):
    """The reference arm: the paper publishes no code, so the FP64 oracle as it stands
    runs on every usable host core (one process per core, each over its own block of
    C_sigma) on the same workload, restarts and initial points; a step is one round of
    all processes at once (~3 s each)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    make, R = WORKLOADS[args.workload]
    inst = make()
    a, b = W.initial_point(inst, R, seed=replica_seed(0))
    sigma = inst.scale / (0.1 * 10)
    cores, model = host_cpu()
    budget = 3.0
    _, k1, _, _ = oracle_sample_rate(inst, R, a, b, sigma, budget)
    per = max(64, 2 * k1)
    pool = OraclePool(inst, R, a, b, sigma, cores, per)
    try:
        for _ in range(args.warmup):
            pool.run(1.0)
        rates, ks, secs = [], [], 0.0
        for _ in range(args.steps):
            r, k, dt = pool.run(budget)
            rates.append(r)
            ks.append(k)
            secs += dt
    finally:
        pool.close()
    value = float(np.mean(rates))
    sample = (f"{cores} processes, each over its own block of {per} constraints of C_sigma x {R} restarts, "
              f"~{budget:.0f} s of FP64 numpy forward+adjoint per step ({int(np.mean(ks))} constraints per step), "
              f"{inst.name}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": inst.name, "restarts": R, "n_vars": inst.n_bool + inst.n_real,
                       "n_cons": inst.n_cons},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": model},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def fused_roofline(info, inst, R, nodes, fused_ms, launch, workload, peaks, peak_kind, n_sm):
    """Roofline of the fused forward + adjoint kernel against both roofs it could hit.

    Work per launch: 10 FP32 flops per decision-node visit (Alg. 3: two FMA; Alg. 4:
    one subtract, one FMA; the adjoint sum: one FMA), against n_sm x 128 FP32 lanes x
    2 flops x the maximum SM clock; and the algorithmic bytes (structure once: 8 B per
    node, 17 B per atom, 8 B per nonzero, 9 B per constraint; state once: w, a and b
    in, the gradients out, the objective) against the measured HBM bandwidth.  The
    reported bound is the roof the kernel is nearer to (the larger fraction).  At the
    FP32 roof the same launch would move its bytes at alg_bytes / (alg_flops /
    alu_peak): the fraction of HBM a fused form of this work can reach at most."""
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    alu_peak = n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12
    alg_flops = 10.0 * nodes * R
    structure = nodes * 8 + info["n_atoms"] * 17 + info["atom_nnz"] * 8 + info["n_obj_cons"] * 9
    state = 4 * R * (info["n_obj_cons"] + 2 * (inst.n_bool + inst.n_real) + 1)
    alg_bytes = structure + state
    sec = fused_ms / 1000.0
    alu = {"achieved": alg_flops / sec / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
           "frac": alg_flops / sec / 1e12 / alu_peak,
           "peak_kind": f"derived: {n_sm} SMs x 128 FP32 lanes x 2 flops (FMA) x {sm_mhz:.0f} MHz"}
    hbm = {"achieved": alg_bytes / sec / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": alg_bytes / sec / 1e9 / peaks["hbm_gbs"], "peak_kind": f"{peak_kind} (copy bandwidth)"}
    cap = alg_bytes / (alg_flops / (alu_peak * 1e12)) / 1e9 / peaks["hbm_gbs"]
    top, bound = (alu, "alu") if alu["frac"] >= hbm["frac"] else (hbm, "hbm")
    traffic, traffic_note = profiled_traffic(workload, R)
    return {"bound": bound, "achieved": top["achieved"], "peak": top["peak"], "unit": top["unit"],
            "frac": top["frac"], "traffic": traffic, "peak_kind": top["peak_kind"],
            "kernel": kernel_name(launch), "kernel_ms": fused_ms, "algorithmic_flops": alg_flops,
            "algorithmic_bytes": alg_bytes, "traffic_source": traffic_note,
            "node_visits_per_s": nodes * R / sec, "alu": alu, "hbm": hbm,
            "hbm_target": {"frac": 0.5, "met": hbm["frac"] >= 0.5, "hbm_frac_at_fp32_roof": cap,
                           "note": "at 10 FP32 flops per node visit the FP32 roof caps a fused form of this "
                                   "work at hbm_frac_at_fp32_roof of HBM bandwidth"}}


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
    S = Solver(P, comp, R, eta=eta, b_scale=inst.scale, t_max=args.iters, sweeps=20, use_graph=True,
               stage_form=args.stage_form)
    S.reset(a0, b0)
    sched = [inst.scale / (0.1 * t) for t in range(1, 21)]
    # autotuned forward + adjoint configuration (fsmt_autotune), then the stage form
    launch = S.tune(sched[0]).as_dict()
    stage_form = S.chosen_stage_form
    stream = torch.cuda.current_stream()
    nodes = info["n_obj_nodes"]

    def step(k):
        S.stage(sched[k % len(sched)], k + 1)

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    S.check_stage_status()
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
    S.check_stage_status()
    # a stage stops early only when every restart has converged: count what ran
    iters_per_step = int(S.iters.max().item())
    ms = max_over_ranks(ms, dev)
    clk = clocks.stop()
    value = whole_job_rate(nodes * R * iters_per_step * args.steps, ws, ms)

    # every stage form timed on the same state: the tuner's own timings (two stages each)
    stage_forms = dict(S.stage_form_ms or {stage_form: ms / args.steps})

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
    d2h = R * 8 + 4  # #Unsat and the objective per restart, and the stage's error bits

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
    roofline = fused_roofline(info, inst, R, nodes, fused_ms, launch, args.workload, peaks, peak_kind,
                              torch.cuda.get_device_properties(dev).multi_processor_count)

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
    if ws > 1 and args.tts_protocol == "first":
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
                       "restart": res["restart"], "stages_run": res["stages_run"], "best_unsat": res["best_unsat"],
                       "rejected_candidates": res["rejected_candidates"], "seed": s}
                if ws > 1:
                    rec["found_here"] = res["sat"]
                if solved:
                    rec["inv_sigma_over_scale"] = round(0.1 * res["stages_run"], 1)
                runs.append(rec)
                del S2
                torch.cuda.empty_cache()
            from paper_2603_22877_b300 import gather_replicas, replica_median
            if ws > 1 and args.tts_protocol == "median":   # every replica's runs, for the median over all
                runs = [dict(r, rank=k) for k, rr in enumerate(gather_replicas(runs)) for r in rr]
            tts[form] = {"median_s_par2": replica_median(runs, args.tts), "solved": sum(r["sat"] for r in runs),
                         "seeds": len(runs), "runs": runs,
                         "protocol": args.tts_protocol if ws > 1 else "median over seeds"}
        if "plain" in tts:
            # same initial points, same schedule: the batched fused form against the plain one,
            # as the ratio of the PAR-2 medians over the (replica, seed) runs both forms made
            par2 = {f: {(r.get("rank", 0), r["seed"]): (r["seconds"] if r["sat"] else 2 * args.tts)
                        for r in tts[f]["runs"]} for f in ("fused", "plain")}
            both = sorted(set(par2["fused"]) & set(par2["plain"]))
            tts["plain_over_fused_median"] = float(np.median([par2["plain"][k] for k in both]) /
                                                   np.median([par2["fused"][k] for k in both]))
            tts["plain_over_fused_per_seed"] = [par2["plain"][k] / par2["fused"][k] for k in both]

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:  # the host baseline runs at N = 1 only
        cpu = cpu_baseline(inst, R, a0, b0, sigma)
    # per stage: parameters, stage start, weight sums; per iteration: iteration
    # start, fused forward+adjoint, one PGD kernel per variable class, convergence
    # test; then round + check: over the chunks for C_sigma, one warp per constraint
    # for the rest (graph iterations past convergence still launch)
    checks = (info["n_chunks"] > 0) + (info["n_chunks"] == 0 or inst.n_cons > info["n_obj_cons"])
    if stage_form == "stage":  # parameters, stage start, weight sums, iteration start, the stage kernel, checks
        launches_per_step = 5 + checks
    elif stage_form == "iteration":  # the same with the stage kernel once per iteration
        launches_per_step = 4 + args.iters + checks
    else:
        launches_per_step = 3 + args.iters * (3 + (inst.n_bool > 0) + (info["n_free_reals"] > 0) +
                                              (info["n_components"] > 0)) + checks
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "restarts": R, "n_vars": inst.n_bool + inst.n_real,
                           "n_bool": inst.n_bool, "n_real": inst.n_real, "n_cons": inst.n_cons,
                           "n_obj_cons": info["n_obj_cons"], "n_obj_nodes": nodes, "atoms": inst.n_atoms,
                           "iters_per_step": iters_per_step, "eta": eta,
                           "form": {"stage": "fused forward + adjoint + PGD, one persistent kernel per stage",
                                    "iteration": "fused forward + adjoint + PGD, one persistent kernel per iteration",
                                    "launches": "fused forward + adjoint, PGD kernels, separate launches per "
                                                "iteration"}[stage_form] + ", CUDA graph",
                           "stage_form": stage_form,
                           "l2": "inputs larger than L2 (diagrams + weights > 126 MB)",
                           "compile_s": compile_s, "upload_s": upload_s, "parallelism": f"replicas x{ws}",
                           "launch": launch},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches_per_step * args.steps, "clocks": clk, "stage_forms_ms": stage_forms,
                "plain": plain,
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
