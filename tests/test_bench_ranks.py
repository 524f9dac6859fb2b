"""bench.py's multi-rank logic on CPU: two gloo ranks (spawned processes)
exercise the process-group setup from the torchrun environment, the barrier,
the max-over-ranks step time and the sum of units over ranks that the
replicated benchmark reports (value = all ranks' units / slowest rank's
time)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), BENCH_BACKEND="gloo")
    import torch.distributed as dist

    import bench
    d, r, w = bench._dist()
    bench._barrier(d)
    slowest = bench._max_over_ranks(d, 1.5 + rank)        # per-rank step times
    units = bench._sum_over_ranks(d, 1000.0 * (rank + 1))  # per-rank units
    q.put((r, w, slowest, units))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_replicated_bench():
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
    assert [o[0] for o in out] == [0, 1]
    for _, w, slowest, units in out:
        assert w == 2
        assert slowest == 2.5          # max over ranks, seen by every rank
        assert units == 3000.0         # sum over ranks
