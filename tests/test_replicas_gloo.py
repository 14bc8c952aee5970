"""The multi-GPU path of bench.py is "replicas only": every rank runs the
whole workload, the job's time is the slowest rank's, and the value is the
units of all ranks over that time.  Checked here with two gloo ranks on CPU
(the GPU runs use NCCL through the same functions)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local = [120.0, 75.5][rank]
    slow = bench.slowest_ms(local, ws, "cpu")
    value = bench.replica_value(1000, 4, ws, slow)
    q.put((rank, slow, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, value in out:
        assert slow == 120.0
        assert value == pytest.approx(2 * 1000 * 4 / 0.120)


def test_single_replica_is_local():
    import bench
    assert bench.slowest_ms(42.0, 1, "cpu") == 42.0
    assert bench.replica_value(10, 2, 1, 1000.0) == pytest.approx(20.0)
