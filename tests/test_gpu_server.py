"""The served request loop: results are the same alone and in the mix.

One request stream (new trees and re-touches of earlier ones, arriving within
a few tens of milliseconds) runs through a 4-slot server with a small device
budget (so trees are evicted and come back), and through the sequential mode
(one request at a time, nothing resident).  Each request deep-copies its tree,
applies position += 0.5*velocity and copies back, so after the stream a tree
has been updated once per request on it: both runs must leave every host tree
bit-identical to the oracle doing the same requests one by one."""
import random

import pytest
import torch

import oracle
import treegen as tg
from bump import BumpAllocator
import paper_1906_01128_b300 as dc

pytestmark = pytest.mark.gpu


def request_stream(nkeys, nreq, seed, span_s):
    rng = random.Random(seed)
    seen, reqs, nxt = [], [], 0
    for i in range(nreq):
        if seen and (rng.random() < 0.3 or nxt >= nkeys):
            k, retouch = rng.choice(seen), 1
        else:
            k, retouch, nxt = nxt, 0, nxt + 1
            seen.append(k)
        reqs.append((k, rng.uniform(0, span_s), retouch))
    reqs.sort(key=lambda r: r[1])
    return reqs


def oracle_replay(trees, reqs):
    s = trees[0].schema
    op = oracle.Op()
    for k, _, _ in reqs:
        cp = oracle.deep_copy(s, trees[k].root)
        oracle.update(s, cp.root, op)
        oracle.copy_back(s, cp.root, trees[k].root, op)


@pytest.mark.parametrize("slots,budget_mb", [(4, 6), (4, 256), (8, 64)])
def test_same_results_alone_and_in_the_mix(slots, budget_mb):
    nkeys, nreq = 48, 160
    mk = lambda: tg.batched(nkeys, seed=7, t_min=16 << 10, t_max=512 << 10)  # noqa: E731
    mix, alone, ref = mk(), mk(), mk()
    s = mix[0].schema
    reqs = request_stream(nkeys, nreq, seed=slots * 100 + budget_mb, span_s=0.05)
    pool = torch.empty(budget_mb << 20, dtype=torch.uint8, device="cuda")
    srv = dc.Server(s, pool, pinned_bytes=budget_mb << 20, slots=slots)
    lat = srv.run([(k, mix[k].root, a, r) for k, a, r in reqs])
    st = srv.stats
    assert st["served"] == nreq and st["failed"] == 0 and min(lat) >= 0
    if budget_mb == 6:
        assert st["evictions"] > 0  # a small budget: trees left and came back
    assert st["resident_hits"] > 0
    srv.destroy()
    seq = dc.Server(s, pool, pinned_bytes=budget_mb << 20, slots=1, flags=dc.SERVER_SEQUENTIAL)
    seq.run([(k, alone[k].root, a, r) for k, a, r in reqs])
    assert seq.stats["resident_hits"] == 0
    seq.destroy()
    oracle_replay(ref, reqs)
    for k in range(nkeys):
        ok, msg = oracle.trees_equal(s, mix[k].root, ref[k].root)
        assert ok, ("mix", k, msg)
        ok, msg = oracle.trees_equal(s, alone[k].root, ref[k].root)
        assert ok, ("alone", k, msg)


def test_served_trees_staged_by_host_spans():
    """Trees of 1,244 blocks with 40-byte arrays: each request's plan stages its deep copy by host
    spans, into the pinned staging the server lends it; with evictions and re-touches every host
    tree still ends bit-identical to the oracle's replay."""
    nkeys, nreq = 32, 100
    # the mix's trees from one bump buffer, so that each lies together in host memory (in a
    # process whose heap is fragmented, malloc scatters small blocks and the rule stages block by block)
    bump = BumpAllocator(nkeys * (128 << 10))
    mix = [tg.node_tree(4, 8, 10, seed=300 + k, alloc=bump.alloc) for k in range(nkeys)]
    ref = [tg.node_tree(4, 8, 10, seed=300 + k) for k in range(nkeys)]
    s = mix[0].schema
    p = dc.Plan(s, mix[0].root)
    assert p.info["staging_bytes"] > 0 and p.info["nblocks"] == 1244
    p.destroy()
    reqs = request_stream(nkeys, nreq, seed=11, span_s=0.05)
    pool = torch.empty(4 << 20, dtype=torch.uint8, device="cuda")
    srv = dc.Server(s, pool, pinned_bytes=16 << 20, slots=4)
    srv.run([(k, mix[k].root, a, r) for k, a, r in reqs])
    st = srv.stats
    assert st["served"] == nreq and st["failed"] == 0 and st["evictions"] > 0 and st["resident_hits"] > 0
    srv.destroy()
    oracle_replay(ref, reqs)
    for k in range(nkeys):
        ok, msg = oracle.trees_equal(s, mix[k].root, ref[k].root)
        assert ok, (k, msg)


def test_request_larger_than_the_budget_fails_alone():
    small = tg.batched(6, seed=3, t_min=16 << 10, t_max=64 << 10)
    big = tg.node_tree(2, 4, 1 << 20, seed=5)  # ~40 MB
    s = big.schema
    pool = torch.empty(8 << 20, dtype=torch.uint8, device="cuda")
    srv = dc.Server(s, pool, pinned_bytes=64 << 20, slots=2)
    reqs = [(i, t.root, 0.001 * i, 0) for i, t in enumerate(small)] + [(99, big.root, 0.002, 0)]
    with pytest.raises(dc.DcError) as e:
        srv.run(reqs)
    assert e.value.name == "DC_EBUDGET"
    st = srv.stats
    assert st["served"] == len(small) and st["failed"] == 1
    srv.destroy()
