"""The multi-GPU path of the benchmark runs independent replicas (one per rank, no
collective on the data path) and reduces only the timings: a world_size-2 gloo run on
the CPU checks that reduction and the whole-job throughput."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as tdist
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [10.0 + 5.0 * rank, 3.0 - rank, 7.0]
    got = bench.reduce_max(ms, "cpu")
    val = bench.weak_scaling_value(1000.0, 4, world, got[0])
    out.put((rank, got, val))
    tdist.barrier()
    tdist.destroy_process_group()


def test_replica_timings_reduce_to_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, val in res:
        assert got == [15.0, 3.0, 7.0]
        assert val == pytest.approx(1000.0 * 4 * 2 / 15e-3)


def test_single_process_is_a_no_op():
    import bench
    assert bench.reduce_max([1.0, 2.0], "cpu") == [1.0, 2.0]
