"""The N > 1 bench path on CPU: two gloo ranks each build their own tree (the
workload's seed shifted by the rank), plan it, and the whole-job throughput
uses the slowest rank's time.  No GPU: the data path has no collective, so the
only exchange is this max over ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    import treegen as tg
    import paper_1906_01128_b300 as dc
    seed = bench.rank_seed("tiny", rank)
    t = tg.node_tree(*tg.WORKLOADS["tiny"][:4], seed=seed)
    plan = dc.Plan(t.schema, t.root)
    c = oracle.count(t.schema, t.root)
    assert plan.info["payload_bytes"] == c["payload_bytes"] == t.payload_bytes
    t_local = 0.5 + rank  # a stand-in step time: rank 1 is the slowest
    value, t_max = bench.aggregate(t.payload_bytes, 4, t_local, world, dist)
    out[rank] = (seed, value, t_max, t.payload_bytes)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    seeds = {res[r][0] for r in range(world)}
    assert len(seeds) == world  # independent trees per rank
    for r in range(world):
        seed, value, t_max, payload = res[r]
        assert t_max == pytest.approx(1.5)  # the slowest rank's time
        assert value == pytest.approx(payload * world * 4 / 1.5 / 1e9)


def _lpt_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import bench
    import treegen as tg
    import paper_1906_01128_b300 as dc
    ranks = bench.Ranks(torch, world)  # gloo: no GPU here
    specs = tg.batched_specs(60, seed=9, t_max=256 << 10)
    part, loads = dc.partition_by_bytes([sp.bytes for sp in specs], world)
    mine = [sp for sp, k in zip(specs, part) if k == rank]
    trees = [sp.build() for sp in mine]
    assert all(t.payload_bytes == sp.bytes for t, sp in zip(trees, mine))  # sizes counted without building
    out[rank] = (part, loads, [sp.index for sp in mine], ranks.sum(len(mine)), ranks.sum(sum(sp.bytes for sp in mine)),
                 ranks.max(float(rank)))
    ranks.barrier()
    ranks.close()


def test_two_gloo_ranks_take_disjoint_lpt_shares():
    """The batched bench path with N ranks: every rank draws the same tree sizes,
    computes the same greedy-LPT assignment on its own, and builds only its
    share; together the shares cover every tree once, with byte totals that
    differ by at most the largest tree."""
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_lpt_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] and res[0][1] == res[1][1]  # the same assignment on both ranks
    assert sorted(res[0][2] + res[1][2]) == list(range(60))
    loads = res[0][1]
    import treegen as tg
    sizes = [sp.bytes for sp in tg.batched_specs(60, seed=9, t_max=256 << 10)]
    assert sum(loads) == sum(sizes) and max(loads) - min(loads) <= max(sizes)
    for r in range(world):
        assert res[r][3] == 60 and res[r][4] == sum(sizes) and res[r][5] == world - 1
