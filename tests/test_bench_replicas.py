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
