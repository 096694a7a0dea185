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
