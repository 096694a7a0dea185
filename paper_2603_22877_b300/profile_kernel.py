"""Launches the forward + adjoint kernels a few times on one workload, for
profilers: python -m paper_2603_22877_b300.profile_kernel --workload NAME --launches N
With --stages N it runs N annealing stages instead (the autotuned configuration,
20 PGD iterations each, from a captured CUDA graph), for launch lists of a stage.
The autotuner's choice is printed as an index into the instance's launch
configurations; --config INDEX pins that one instead of tuning, so that a run under
a profiler (where the tuner's timings are distorted) uses the kernels a plain run
chose.  --form picks how a stage runs (separate launches per iteration, one
persistent kernel for the stage, or that kernel once per iteration); with --trace
the persistent kernel records the global timer as each of its grid barriers opens,
and the mean forward + adjoint and PGD phase times are printed with the stages'
CUDA-event time.

Workloads are the seeded synthetic instances of the `workloads` package; the
smaller variants keep a profiler capture short."""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import instances as W  # noqa: E402

CASES = {
    "large_scheduling": (lambda: W.large_scheduling(1005), 512),
    "large_scheduling_400": (lambda: W.large_scheduling(1005, n_jobs=400), 512),
    "placement2d": (lambda: W.placement2d(1003), 1024),
    "placement2d_200": (lambda: W.placement2d(1003, 200), 1024),
    "jobshop": (lambda: W.jobshop(1002), 256),
    "uneven_batch": (lambda: W.concat(W.uneven_batch(1004), "uneven_batch"), 32),
}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="large_scheduling_400", choices=list(CASES))
    p.add_argument("--launches", type=int, default=3)
    p.add_argument("--plain", action="store_true")
    p.add_argument("--stages", type=int, default=0, help="annealing stages to run instead of bare launches")
    p.add_argument("--config", type=int, default=-1, help="with --stages: pin this launch configuration (index)")
    p.add_argument("--form", default="stage", choices=["launches", "stage", "iteration"])
    p.add_argument("--trace", action="store_true", help="with --stages: per-phase times of the persistent kernel")
    args = p.parse_args()
    import torch
    from paper_2603_22877_b300 import build
    from paper_2603_22877_b300.engine import Problem
    build.build()
    make, R = CASES[args.workload]
    inst = make()
    P = Problem.from_instance(inst)
    comp = P.compile().upload()
    a, b = W.initial_point(inst, R, seed=7)
    da = torch.from_numpy(a).cuda()
    db = torch.from_numpy(b).cuda()
    dw = torch.ones((inst.n_cons, R), device="cuda")
    ga, gb = torch.zeros_like(da), torch.zeros_like(db)
    obj = torch.zeros(R, device="cuda")
    sigma = inst.scale
    if args.stages > 0:
        from paper_2603_22877_b300 import Solver
        S = Solver(P, comp, R, eta=0.02, b_scale=inst.scale, t_max=20, sweeps=20, use_graph=True,
                   stage_form=args.form)
        S.reset(a, b)
        sched = [inst.scale / (0.1 * t) for t in range(1, 21)]
        cfgs = comp.launch_configs(R)
        key = lambda c: (c.variant, c.restarts_per_lane, c.staged_reals, c.warps)
        if args.config >= 0:
            comp.select_config(R, cfgs[args.config])
            idx = args.config
        else:
            best = S.tune(sched[0])
            idx = [key(c) for c in cfgs].index(key(best))
        persistent = S.persistent and comp.stage_form(R)
        trace = None
        if args.trace and persistent:
            trace = torch.zeros(1 + 2 * S.t_max, dtype=torch.int64, device="cuda")
            comp.stage_trace(trace)
        S.stage(sched[0], 1)  # graph capture and first use outside the timed stages
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        phases = []
        e0.record()
        for k in range(args.stages):
            S.stage(sched[k % len(sched)], k + 1)
            if trace is not None:  # the stage's phase boundaries, read after it ends
                t = trace.cpu().numpy().astype(np.float64)
                n = int(S.iters.max())
                ends = t[1:1 + 2 * n]
                starts = np.concatenate([[t[0]], ends[1::2][:-1]])
                phases.append(((ends[0::2] - starts) / 1e6, (ends[1::2] - ends[0::2]) / 1e6))
        e1.record()
        torch.cuda.synchronize()
        S.check_stage_status()
        print("stages", args.stages, "iters", int(S.iters.max()), "n_unsat min", int(S.n_unsat.min()),
              "config", idx, cfgs[idx].as_dict(), "form", S.chosen_stage_form)
        print("ms per stage (events%s) %.3f" % (", trace reads between stages" if trace is not None else "",
                                                e0.elapsed_time(e1) / args.stages))
        if phases:
            fa = np.concatenate([p[0] for p in phases[1:] or phases])
            pg = np.concatenate([p[1] for p in phases[1:] or phases])
            print("persistent kernel, ms per iteration: forward + adjoint %.4f, PGD + epsilon test %.4f"
                  % (fa.mean(), pg.mean()))
            comp.stage_trace(None)
        return
    work = torch.empty(comp.plain_work(R), device="cuda") if args.plain else None
    for _ in range(args.launches):
        if args.plain:
            comp.forward_plain(R, sigma, dw, da, db, work, obj=obj)
            comp.adjoint_plain(R, sigma, dw, da, db, work, ga, gb)
        else:
            comp.adjoint(R, sigma, dw, da, db, ga, gb, obj=obj)
    torch.cuda.synchronize()
    print("nodes", comp.info["n_obj_nodes"], "R", R, "obj[0]", float(obj[0]))


if __name__ == "__main__":
    main()
