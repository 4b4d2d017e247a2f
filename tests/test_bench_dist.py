"""Host logic of the multi-rank bench (replicas, slowest-rank timing) on two
gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank  # rank 1 is slower
    slow = bench.max_over_ranks(ms, dist, device="cpu")
    rate = bench.whole_job_rate(world, 1.0e9, slow)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, slow, rate))


def test_two_rank_replica_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slow, rate in res:
        assert slow == 15.0  # the slowest rank's time, on every rank
        assert rate == pytest.approx(2 * 1.0e9 / 0.015)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_rate(1, 3.0e9, 1000.0) == pytest.approx(3.0e9)


def test_cpu_baseline_threads_and_single_core():
    """The CPU-baseline leg reports the oracle's thread count, a one-thread
    rate below the all-thread one (or equal on one core), and leaves the
    oracle's thread count as it found it."""
    import bench
    from oracle import oracle as orc
    before = orc.threads()
    r = bench.cpu_baseline(seconds=1.0)
    assert orc.threads() == before == r["cores"]
    assert r["kind"] == "oracle" and r["value"] > 0 and r["single_core_value"] > 0
    if r["cores"] > 1:
        assert r["single_core_value"] < r["value"]
    assert orc.threads(1) == 1
    orc.threads(before)
