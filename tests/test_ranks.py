"""Multi-rank host logic of the batched workload (one process per GPU, no data exchange):
instance blocks per rank and the timing reductions, run as two gloo processes on the CPU."""
import os
import socket

import pytest

from paper_2303_15861_gb300 import ranks
from paper_2303_15861_gb300 import workloads as W


@pytest.mark.parametrize("count,world", [(0, 1), (1, 1), (512, 1), (1024, 2), (7, 3), (3, 8), (4096, 8), (513, 4)])
def test_shard_covers_every_unit_once_and_balances(count, world):
    blocks = [ranks.shard(count, r, world) for r in range(world)]
    seen = [i for lo, hi in blocks for i in range(lo, hi)]
    assert seen == list(range(count))
    sizes = [hi - lo for lo, hi in blocks]
    assert max(sizes) - min(sizes) <= 1


def test_shard_rejects_bad_ranks():
    with pytest.raises(ValueError):
        ranks.shard(8, 2, 2)
    with pytest.raises(ValueError):
        ranks.shard(8, 0, 0)


def test_selected_instances_equal_the_full_draw():
    """A rank's block holds exactly the instances of the global draw at those indices."""
    full = W.config4(count=6, m=2)
    part = W.config4(count=6, m=2, select=range(3, 6))
    for a, b in zip(full[3:], part):
        assert a.dims == b.dims and a.b == b.b
        assert (a.a_nodes == b.a_nodes).all() and (a.u0 == b.u0).all()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = ranks.rank_env()
    count = 16 * w
    lo, hi = ranks.shard(count, r, w)
    draws = W.config4_draws(count)
    dof = sum(d["n"] ** 2 for d in draws[lo:hi])
    blocks = [None] * w
    dist.all_gather_object(blocks, (lo, hi))
    total = ranks.reduce_scalar(dof, "sum", dist, "cpu")
    slowest = ranks.reduce_scalar(1.0 + r, "max", dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((r, blocks, total, slowest, sum(d["n"] ** 2 for d in draws)))


def test_two_gloo_ranks_cover_the_draw_and_reduce_timings():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, blocks, total, slowest, expect in res:
        assert blocks == [(0, 16), (16, 32)]
        assert total == expect                  # the DOF of every rank's block, summed
        assert slowest == 2.0                   # the slowest rank's time
