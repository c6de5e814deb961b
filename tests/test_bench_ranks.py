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


def test_kernel_hash_ignores_comments_only():
    """The hash tying a profile summary to the kernel code skips comments and blank lines and
    keeps everything else, string literals included."""
    import bench
    a = "int f(int x) {  // first\n  /* block\n comment */ return x + 1;\n}\n"
    b = "int f(int x) {\n\n  return x + 1;   // other words\n}\n"
    c = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench.code_text(a) == bench.code_text(b) != bench.code_text(c)
    assert "//kept" in bench.code_text('const char* s = "//kept"; // dropped\n')
    assert "dropped" not in bench.code_text('const char* s = "//kept"; // dropped\n')
