"""The N > 1 bench path on CPU: two gloo ranks agree on the slowest rank's
time (max over ranks) and the whole-job value is N replicas' throughput."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                      # rank 1 is slower
    m = bench.max_over_ranks(ms, world, device="cpu")
    q.put((rank, m, bench.job_value(20 / (m * 1e-3), world)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling_value():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    assert abs(out[0][2] - 2 * 20 / 0.015) < 1e-9
