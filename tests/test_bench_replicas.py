"""Host logic of bench.py under torchrun: every rank is an independent replica
(own restart seeds), the timed region is the slowest rank's, and the value is the
whole job's.  Two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = 100.0 + 50.0 * rank  # rank 1 is the slower one
        m = bench.max_over_ranks(ms)
        out[rank] = (bench.replica_seed(rank), m, bench.whole_job_rate(1000, ws, m))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas():
    ws, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    seeds = {res[r][0] for r in range(ws)}
    assert len(seeds) == ws  # independent initial points per replica
    for r in range(ws):
        assert res[r][1] == pytest.approx(150.0)  # every rank reports the slowest time
        assert res[r][2] == pytest.approx(1000 * ws / 0.150)  # units of all ranks / max time


def test_without_process_group_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_rate(10, 1, 1000.0) == pytest.approx(10.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"])
    bench.reference_arm(bench.parse())
    assert capsys.readouterr().out == ""  # the other ranks exit without work


def _fake_solver(sat_stage, R=4):
    """A Solver whose stages are scripted on the host: restart 1 reaches #Unsat = 0 at
    stage sat_stage (never when None) and verifies; no device is touched."""
    import sys
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    from paper_2603_22877_b300 import Solver

    class Fake(Solver):
        def __init__(self):
            self.R = R
            self.n_unsat = torch.full((R,), 3, dtype=torch.int32)
            self.iters = torch.full((R,), 7, dtype=torch.int32)
            self.gnorm2 = torch.full((R,), 0.25)
            self.obj = torch.full((R,), -1.0)
            self.form, self._form_code = "fused", 1  # a persistent stage form
            self.ctl = torch.zeros(4, dtype=torch.int32)  # no error bits: every stage completed
            self.calls = 0

        def stage(self, sigma, t):
            self.calls += 1
            self.obj[0] = -1.0 - t
            if sat_stage is not None and t >= sat_stage:
                self.n_unsat[1] = 0

        def verify_restart(self, r):
            return True, np.ones(1, np.int8), np.zeros(1)
    return Fake()


def _anneal_rank(rank, ws, port, out, sat_stages, limits):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2603_22877_b300 import max_over_replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        S = _fake_solver(sat_stages[rank])
        res = S.anneal([1.0] * 10, time_limit=limits[rank], share=max_over_replicas("cpu"))
        out[rank] = (res["sat"], res["stopped_by_peer"], res["stages_run"], S.calls)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("sat_stages,limits,expect", [
    ((3, None), (None, None), {0: (True, False, 3, 3), 1: (False, True, 3, 3)}),
    ((None, 5), (None, None), {0: (False, True, 5, 5), 1: (True, False, 5, 5)}),
    ((None, None), (None, 0.0), {0: (False, False, 1, 1), 1: (False, False, 1, 1)}),
    ((None, None), (None, None), {0: (False, False, 10, 10), 1: (False, False, 10, 10)}),
])
def test_replicas_stop_together(sat_stages, limits, expect):
    """Restart replicas share one [SAT verified, out of time] flag per stage (Alg. 2 run
    on every rank with its own seeds): all ranks stop after the first stage at which any
    of them verified SAT or ran out of time, so no rank waits in a collective alone."""
    ws, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_anneal_rank, args=(ws, port, out, sat_stages, limits), nprocs=ws, join=True)
        res = dict(out)
    assert res == expect


def test_anneal_without_share_is_unchanged():
    S = _fake_solver(4)
    res = S.anneal([1.0] * 10)
    assert res["sat"] and res["stage"] == 4 and res["stages_run"] == 4 and not res["stopped_by_peer"]
    S = _fake_solver(None)
    res = S.anneal([1.0] * 6)
    assert not res["sat"] and res["stages_run"] == 6 and res["best_unsat"] == 3


def test_anneal_log_writes_one_json_line_per_stage(tmp_path):
    """The per-stage record of Solver.anneal (#Unsat statistics, iterations, ||g||^2,
    best objective) through jsonl_log; a non-finite restart is left out of the
    statistics and counted."""
    import json
    import sys
    sys.path.insert(0, ROOT)
    from paper_2603_22877_b300 import jsonl_log
    S = _fake_solver(3)
    S.n_unsat[2] = -2 ** 31 + 4                            # restart 2 marked non-finite
    S.obj[2] = float("nan")
    path = tmp_path / "trace.jsonl"
    log = jsonl_log(str(path))
    res = S.anneal([2.0, 1.0, 0.5, 0.25], log=log)
    log.close()
    assert res["sat"] and res["stage"] == 3
    recs = [json.loads(line) for line in path.read_text().splitlines()]
    assert [r["stage"] for r in recs] == [1, 2, 3]
    assert [r["sigma"] for r in recs] == [2.0, 1.0, 0.5]
    assert [r["min_unsat"] for r in recs] == [3, 3, 0]
    assert [r["at_zero"] for r in recs] == [0, 0, 1]
    assert all(r["nonfinite"] == 1 and r["mean_iters"] == 7.0 and r["median_gnorm2"] == 0.25 for r in recs)
    assert [r["best_obj"] for r in recs] == [-2.0, -3.0, -4.0]
    assert recs[0]["median_unsat"] == 3.0


def test_constraint_slice_keeps_each_constraints_contribution():
    """bench.constraint_slice (a worker's share of the input for the all-core oracle
    timing) renumbers the atoms it keeps; every kept constraint must contribute to
    C_sigma and its gradient exactly as in the whole instance."""
    import sys
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from oracle import objective as OBJ
    from workloads import instances as W
    inst = W.large_scheduling(1005, 16, 30, 6, 4, 5)
    R = 6
    a, b = W.initial_point(inst, R, seed=2)
    a, b = a.astype(np.float64), b.astype(np.float64)
    oc = OBJ.objective_constraints(inst)
    cons = oc[7:40:3]
    sub = bench.constraint_slice(inst, cons)
    assert sub.n_cons == len(cons) and sub.n_bool == inst.n_bool and sub.n_real == inst.n_real
    D, Ds = OBJ.Diagrams(inst), OBJ.Diagrams(sub)
    sigma = inst.scale / 0.8
    for j, c in enumerate(cons):
        o1, cop1, ga1, gb1 = OBJ.constraint_contrib(inst, D, c, a, b, np.ones(R), sigma)
        o2, cop2, ga2, gb2 = OBJ.constraint_contrib(sub, Ds, j, a, b, np.ones(R), sigma)
        np.testing.assert_array_equal(o1, o2)
        assert ga1.keys() == ga2.keys() and gb1.keys() == gb2.keys()
        for k in ga1:
            np.testing.assert_array_equal(ga1[k], ga2[k])
        for k in gb1:
            np.testing.assert_array_equal(gb1[k], gb2[k])


def test_oracle_pool_times_every_worker():
    """The all-core oracle timing runs one spawned process per worker over its own
    block and sums their rates; two workers on a small instance."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from workloads import instances as W
    inst = W.jobshop(1002, 8, 4)
    R = 16
    a, b = W.initial_point(inst, R, seed=1)
    pool = bench.OraclePool(inst, R, a, b, inst.scale, 2, 40)
    try:
        rate, k, dt = pool.run(0.5)
    finally:
        pool.close()
    assert rate > 0 and k > 0 and 0.4 < dt < 5.0
    cores, model = bench.host_cpu()
    assert cores >= 1 and isinstance(model, str)


def _median_rank(rank, ws, port, out, sat_stages):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2603_22877_b300 import gather_replicas, replica_median
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        S = _fake_solver(sat_stages[rank])
        res = S.anneal([1.0] * 8)                      # no shared flag: independent replicas
        runs = gather_replicas([{"sat": res["sat"], "seconds": float(res["stages_run"]), "calls": S.calls}])
        allr = [r for rr in runs for r in rr]
        out[rank] = (S.calls, [r["calls"] for r in allr], replica_median(allr, limit=100.0))
    finally:
        dist.destroy_process_group()


def test_independent_replicas_report_the_median():
    """The paper's protocol (Methods, experimental setup): replicas run independently,
    each to its own exactly verified SAT or its limit, and the median over replicas is
    reported (PAR-2: a miss counts twice the limit).  Three gloo ranks: SAT at stage 2,
    at stage 6, and never (8 stages run, a miss); each rank runs its own stages only,
    every rank sees all three records, and the median is the stage-6 replica's time."""
    ws, port = 3, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_median_rank, args=(ws, port, out, (2, 6, None)), nprocs=ws, join=True)
        res = dict(out)
    assert [res[r][0] for r in range(ws)] == [2, 6, 8]
    for r in range(ws):
        assert res[r][1] == [2, 6, 8] and res[r][2] == 6.0


def test_replica_median_scores_misses_as_par2():
    import sys
    sys.path.insert(0, ROOT)
    from paper_2603_22877_b300 import replica_median
    runs = [{"sat": True, "seconds": 3.0}, {"sat": False, "seconds": 50.0}, {"sat": False, "seconds": 50.0}]
    assert replica_median(runs, 50.0) == 100.0
    assert replica_median(runs[:1] + [{"sat": True, "seconds": 5.0}], 50.0) == 4.0
