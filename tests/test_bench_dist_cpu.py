"""The multi-GPU path of bench.py is replicas (no data exchange): each rank
times its own copy of the workload, the job time is the max over ranks and the
value counts every rank's pixels.  Checked here with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    m = bench.reduce_max_ms(10.0 + 5.0 * rank)
    q.put((rank, m, bench.whole_job_value(1000.0, 4, m, world), bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v, env in got:
        assert m == 15.0
        assert abs(v - 2 * 1000.0 * 4 / 15e-3 / 1e6) < 1e-9
        assert env[0] == rank and env[1] == 2


def test_single_process_helpers():
    import bench
    assert bench.reduce_max_ms(3.5) == 3.5
    assert abs(bench.whole_job_value(2e6, 10, 100.0, 1) - 200.0) < 1e-9
