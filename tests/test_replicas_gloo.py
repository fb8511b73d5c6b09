"""The multi-rank host logic (replicas, sharded batches, max-over-ranks timing)
on two CPU ranks over gloo."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1912_09240_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, work, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    try:
        ws, r, local = replicas.rank_env()
        dist.init_process_group("gloo", rank=r, world_size=ws)
        dist.barrier()
        t_max = replicas.max_over_ranks(10.0 + 5.0 * r, dist)
        total = replicas.sum_over_ranks(100.0 * (r + 1), dist)
        mine = replicas.shard(work, r, ws)
        gathered = [None] * ws
        dist.all_gather_object(gathered, mine)
        dist.barrier()
        dist.destroy_process_group()
        q.put((r, ws, local, t_max, total, mine, gathered))
    except Exception as e:  # pragma: no cover - reported to the parent
        q.put((rank, "error", repr(e)))


@pytest.mark.parametrize("world", [2, 3])
def test_ranks_agree_on_time_and_partition(world):
    work = [float(w) for w in (5, 1, 9, 3, 3, 7, 2, 8, 6, 4, 1, 1)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, work, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort(key=lambda t: t[0])
    for r, res in enumerate(out):
        assert res[1] != "error", res
        rank, ws, local, t_max, total, mine, gathered = res
        assert (rank, ws, local) == (r, world, r)
        assert t_max == 10.0 + 5.0 * (world - 1)                 # the slowest rank's time
        assert total == 100.0 * world * (world + 1) / 2
        assert mine == replicas.shard(work, r, world)           # no communication needed
    # every rank computed the same partition: disjoint shards covering all items
    shards = out[0][6]
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(len(work)))
    loads = [sum(work[i] for i in s) for s in shards]
    assert max(loads) - min(loads) <= max(work)


def test_shard_single_rank_and_errors():
    assert replicas.shard([3.0, 1.0, 2.0], 0, 1) == [0, 1, 2]
    assert replicas.shard([], 0, 2) == []
    with pytest.raises(ValueError):
        replicas.shard([1.0], 2, 2)
    # largest first to the least-loaded rank
    assert replicas.shard([4.0, 3.0, 2.0, 1.0], 0, 2) == [0, 3]
    assert replicas.shard([4.0, 3.0, 2.0, 1.0], 1, 2) == [1, 2]


def test_max_over_ranks_without_process_group():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.sum_over_ranks(2.0) == 2.0
