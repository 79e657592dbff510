"""Multi-GPU runs are independent replicas (the operator has no exchange step
on the data path): the bench aggregates them as the units of all ranks over
the slowest rank's time.  Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    units = [1.0e9, 3.0e9][rank]
    ms = [2.0, 5.0][rank]
    q.put((rank, bench.replica_throughput(units, ms, True)))
    td.destroy_process_group()


def test_two_replicas_sum_units_over_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        value, ms, total = out[r]
        assert ms == 5.0 and total == 4.0e9
        assert value == pytest.approx(4.0e9 / 5.0e-3)


def test_single_process_is_plain_throughput():
    assert bench.replica_throughput(2.0e9, 4.0, False) == (2.0e9 / 4.0e-3, 4.0, 2.0e9)


def test_reference_arm_runs_on_rank_zero_only():
    class A:
        workload = "uniform_gravity"
        periodic = False
        steps = 1
        warmup = 0
        layout = "redundant"
    assert bench.run_reference(A(), 1, 2) is None
