"""The multi-rank logic of bench.py on CPU: two gloo ranks (world size 2, 127.0.0.1).

The benchmark runs one replica per GPU (weak scaling): each rank times its own grid, the job's
time is the slowest rank's (max over ranks), and the reported value is every rank's cells over
that time.  The reference arm does its work on rank 0 only; other ranks return without work.
"""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        b = _bench()
        assert b._dist() == (ws, rank, rank)
        ms = 100.0 + 50.0 * rank  # rank 1 is the slower one
        ms_max = b.max_over_ranks(ms, ws)
        value = b.job_throughput(ws, 4096 * 4096, 10, ms_max)

        class Args:
            steps, warmup = 1, 0

        ref_rc = b.run_reference(Args, ws, rank) if rank != 0 else None
        out[rank] = (ms_max, value, ref_rc)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    ws = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 150.0
    expect = 2 * 4096 * 4096 * 10 / 0.150 / 1e6
    assert abs(out[0][1] - expect) <= 1e-9 * expect and out[0][1] == out[1][1]
    assert out[1][2] == 0  # the reference arm's other ranks exit without work


def test_single_rank_needs_no_process_group():
    b = _bench()
    assert b.max_over_ranks(12.5, 1) == 12.5
    assert b.job_throughput(1, 100, 2, 1.0) == 100 * 2 / 1e-3 / 1e6
