"""The multi-rank bench logic on CPU (gloo, world size 2): replicas only, the
job's time is the slowest rank's, throughput is summed over the replicas, and
only rank 0 runs the reference arm."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    local_ms = 10.0 + 5.0 * rank                       # rank 1 is the slow replica
    ms = bench.max_over_ranks(local_ms, ws, "cpu")
    out[rank] = (ms, bench.whole_job_value(ws, 1 << 20, 4, ms / 1e3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_throughput():
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    expect = 2 * (1 << 20) * 4 / 0.015 / 1e6             # two replicas' points over the slowest time
    assert abs(res[0][1] - expect) < 1e-9 * expect and res[0][1] == res[1][1]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_value(1, 1000, 10, 2.0) == pytest.approx(0.005)


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        workload = "plain_scalar_64"
        gpus = 2
    bench.reference_arm(A())
    assert capsys.readouterr().out == ""
