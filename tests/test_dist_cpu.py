"""Multi-rank host logic of bench.py on CPU: two gloo ranks (replicas, no
data-path collective) agree on the max-over-ranks time, and the whole-job
throughput counts every rank's replica (weak scaling)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    reduce_max = bench.make_reducer(dist, "cpu")
    my_ms = 100.0 + 10.0 * rank           # the slower rank sets the job time
    t = reduce_max(my_ms)
    dist.barrier()
    out.put((r, ws, local, t, bench.whole_job_mlups(1000000, 50, ws, t)))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_scaling():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[3] == 110.0 for r in res)
    # 2 replicas x 1e6 nodes x 50 steps in 110 ms
    assert all(abs(r[4] - 2 * 1e6 * 50 / 0.110 / 1e6) < 1e-9 for r in res)


def test_single_rank_reducer_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.make_reducer(None, "cpu")(3.5) == 3.5
    assert bench.whole_job_mlups(100, 10, 1, 1.0) == pytest.approx(1.0)
