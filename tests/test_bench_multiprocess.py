"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own
replica, agree on the slowest rank's time and on the whole-job value."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [10.0 + 5.0 * rank, 1.0 - 0.5 * rank]  # ms per timed region, e2e seconds
    got = bench.reduce_max(mine)
    q.put((rank, got, bench.job_mlups(128 ** 3, 100, world, got[0] * 1e-3)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_and_count_all_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, got, value in res:
        assert got == [15.0, 1.0]
        assert abs(value - 128 ** 3 * 100 * 2 / 15e-3 / 1e6) < 1e-6
    assert res[0][2] == res[1][2]


def test_single_process_is_a_no_op():
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    assert bench.reduce_max([3.0, 4.0]) == [3.0, 4.0]
    assert abs(bench.job_mlups(100, 10, 1, 2.0) - 500 / 1e6) < 1e-12
