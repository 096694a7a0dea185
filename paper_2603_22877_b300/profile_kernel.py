"""Launches the forward + adjoint kernels a few times on one workload, for
profilers: python -m paper_2603_22877_b300.profile_kernel --workload NAME --launches N

Workloads are the seeded synthetic instances of the `workloads` package; the
smaller variants keep a profiler capture short."""
import argparse
import os
import sys

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
