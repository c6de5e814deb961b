"""The multi-rank benchmark path on CPU: two gloo ranks (replicas) agree on the slowest
rank's time and report whole-job throughput; each rank solves different seeds."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist   # noqa: E402
import torch.multiprocessing as mp   # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = [1000.0, 2500.0][rank]
    mx = bench.max_over_ranks(ms, ws)
    value = bench.whole_job_throughput(10, ws, mx)
    out[rank] = (mx, value, bench.rank_seeds(rank, 3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    (m0, v0, s0), (m1, v1, s1) = out[0], out[1]
    assert m0 == m1 == 2500.0
    assert v0 == v1 == pytest.approx(2 * 10 / 2.5)
    assert not set(s0) & set(s1)
