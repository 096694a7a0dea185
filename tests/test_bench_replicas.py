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
            self.calls = 0

        def stage(self, sigma, t):
            self.calls += 1
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
