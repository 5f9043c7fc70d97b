"""Multi-rank host logic of bench.py on CPU: two gloo ranks.

Units shard across ranks with no collective on the data path; the only
collectives are the report's reductions (template-seconds summed over ranks,
time the slowest rank's), checked here with uneven per-rank work.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bins = bench.shard_bins(7, rank, world)
    tpl_s = 1000.0 * (rank + 1) * len(bins)            # uneven work per rank
    secs = 2.0 + rank                                   # rank 1 is the slowest
    rate, t = bench.job_rate(tpl_s, secs, dist, "cpu")
    q.put((rank, bins, rate, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_bins_and_reduce_the_report():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, bins0, rate0, t0), (r1, bins1, rate1, t1) = out
    assert bins0 == [0, 2, 4, 6] and bins1 == [1, 3, 5]
    assert sorted(bins0 + bins1) == list(range(7))      # every bin on exactly one rank
    total = 1000.0 * 1 * 4 + 1000.0 * 2 * 3
    assert t0 == t1 == 3.0                              # the slowest rank's time, on every rank
    assert rate0 == rate1 == pytest.approx(total / 3.0)


def test_one_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.shard_bins(3, 0, 1) == [0, 1, 2]
    assert bench.job_rate(600.0, 2.0, None, "cpu") == (300.0, 2.0)
