"""Host logic of the N>1 path on CPU: two gloo ranks split an instance list
(every instance exactly once, no data exchanged), the timing is the max over
ranks, results gather on rank 0."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2604_05867_b300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    items = [(22, 0.05 + 0.9 * i / 31) for i in range(32)] + [(n, 0.6) for n in (14, 16, 18, 20)]
    mine = shard.shard(items, rank, world)
    t = shard.max_over_ranks(10.0 + rank)
    got = shard.gather_to_rank0(mine)
    if rank == 0:
        q.put((t, got))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    t, got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == 11.0
    flat = [x for part in got for x in part]
    items = [(22, 0.05 + 0.9 * i / 31) for i in range(32)] + [(n, 0.6) for n in (14, 16, 18, 20)]
    assert sorted(flat) == sorted(items) and len(flat) == len(items)
    assert not set(map(tuple, got[0])) & set(map(tuple, got[1]))


def test_shard_is_a_partition():
    from paper_2604_05867_b300 import shard
    items = list(range(37))
    parts = [shard.shard(items, r, 4) for r in range(4)]
    assert sorted(x for p in parts for x in p) == items
    with pytest.raises(ValueError):
        shard.shard(items, 4, 4)


def _grid_worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2604_05867_b300 import inputs, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = {}
    for name, grid in (("batched", inputs.batched_d_grid()), ("large", {26: list(inputs.LARGE_SWEEP_D)})):
        mine = shard.shard_grid(grid, rank, world)
        work = sum(len(ds) << n for n, ds in mine.items())
        out[name] = (mine, shard.max_over_ranks(float(work)))
    got = shard.gather_to_rank0(out)
    if rank == 0:
        q.put(got)
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_config_grids_shard_over_gloo_ranks(world):
    # the batched (64 instances of mixed n) and large (7 instances at n = 26)
    # configurations split over ranks: every (n, d) instance exactly once, and
    # the slowest rank holds at most one large instance more than its share
    import torch.multiprocessing as mp

    from paper_2604_05867_b300 import inputs
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_grid_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for name, grid in (("batched", inputs.batched_d_grid()), ("large", {26: list(inputs.LARGE_SWEEP_D)})):
        flat = sorted((n, d) for part in got for n, ds in part[name][0].items() for d in ds)
        assert flat == sorted((n, d) for n, ds in grid.items() for d in ds)
        total = sum(len(ds) << n for n, ds in grid.items())
        biggest = max(1 << n for n in grid)
        assert got[0][name][1] <= total / world + biggest
