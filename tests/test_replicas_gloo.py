"""The multi-rank path of bench.py on CPU: two gloo ranks exchange their timed-region
lengths, every rank sees the slowest one, and the whole-job rate counts the units of
all ranks over that time (the replicas run with no data-path collective)."""
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


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.replica_barrier(world)
    slowest = bench.replica_max(times[rank], world, "cpu")
    out.put((rank, slowest, bench.whole_job_rate(1000, 3, world, slowest)))
    bench.replica_barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_timed_region():
    world, times = 2, [1.25, 2.5]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, times, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate in res:
        assert slowest == max(times)
        assert rate == pytest.approx(1000 * 3 * world / max(times))


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.replica_max(3.0, 1) == 3.0
    assert bench.whole_job_rate(10, 2, 1, 4.0) == 5.0
