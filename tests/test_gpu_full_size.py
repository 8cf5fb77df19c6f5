"""Parity at the full sizes and in the launch configurations the bench times.

- Batched: the 4,096-tree forest (seed 4, payloads in [16 KiB, 7 MiB]) on a
  DC_PLAN_MAP_HOST forest plan, split chosen by dc_autotune, relocation +
  update in one persistent launch, copy back: every tree's device image right
  after the deep copy, and every host tree after the copy back, against the
  oracle.
- Served: the Poisson stream (2,000 requests/s for 2 s, 30% re-touches,
  payloads in [16 KiB, 64 MiB], seed 5) through 8 slots over a 40 GB device
  pool, as the bench runs it; every host tree afterwards equals the oracle
  doing the same requests one by one.
"""
import pytest
import torch

import oracle
import treegen as tg
import paper_1906_01128_b300 as dc

pytestmark = pytest.mark.gpu


def test_batched_full_size():
    src, ref = tg.batched(4096, seed=4), tg.batched(4096, seed=4)
    s = src[0].schema
    op = dc.Op()
    plan = dc.Plan(s, [t.root for t in src], flags=dc.PLAN_MAP_HOST)
    plan.bind()
    plan.deep_copy()
    plan.autotune(op)
    plan.deep_copy()  # the tuning runs applied the update: start again from the host trees
    plan.sync()
    img, base = plan.image(), plan.device_base
    for i in range(4096):  # every tree's replica in the one arena
        ok, msg, _ = oracle.check_image(s, src[i].root, img, base, plan.root_offset(i))
        assert ok, (i, msg)
    del img
    plan.relocate_update(op)
    plan.copy_back()
    plan.sync()
    oop = oracle.Op()
    for i, (t, r) in enumerate(zip(src, ref)):  # every tree after the copy back
        cp = oracle.deep_copy(s, r.root)
        oracle.update(s, cp.root, oop)
        oracle.copy_back(s, cp.root, r.root, oop)
        ok, msg = oracle.trees_equal(s, t.root, r.root)
        assert ok, (i, msg)
    plan.destroy()


def test_served_full_configuration():
    reqs, nkeys = tg.poisson_requests(2.0, 2000.0, 0.3, seed=5)
    mk = lambda: tg.batched(nkeys, seed=5, t_min=16 << 10, t_max=64 << 20)  # noqa: E731
    src, ref = mk(), mk()
    s = src[0].schema
    pool = torch.empty(40 << 30, dtype=torch.uint8, device="cuda")
    srv = dc.Server(s, pool, pinned_bytes=24 << 30, slots=8)
    lat = srv.run([(k, src[k].root, a, r) for k, a, r in reqs])
    st = srv.stats
    srv.destroy()
    del pool
    assert st["served"] == len(reqs) and st["failed"] == 0 and len(lat) == len(reqs)
    assert st["resident_hits"] > 0
    op = oracle.Op()
    for k, _, _ in reqs:  # the oracle serves the same requests one by one, in arrival order
        cp = oracle.deep_copy(s, ref[k].root)
        oracle.update(s, cp.root, op)
        oracle.copy_back(s, cp.root, ref[k].root, op)
    for k in range(nkeys):
        ok, msg = oracle.trees_equal(s, src[k].root, ref[k].root)
        assert ok, (k, msg)


@pytest.mark.parametrize("name", ["dense", "deep", "reloc_stress"])
def test_bench_step_full_size(name):
    """The bench's step for the single-tree workloads: dc_autotune picks the
    split, then one dc_relocate_update launch (relocation + leaf update) on the
    resident arena, then the copy back; the host tree must equal the oracle's."""
    src, ref = tg.workload(name), tg.workload(name)
    s = src.schema
    op = dc.Op(sel=dc.SEL_CHAIN, path=tg.leaf_path(64)) if name == "deep" else dc.Op()
    oop = oracle.Op(sel=oracle.SEL_CHAIN, path=tg.leaf_path(64)) if name == "deep" else oracle.Op()
    plan = dc.Plan(s, src.root)
    plan.bind()
    plan.deep_copy()
    plan.autotune(op)
    plan.deep_copy()  # the tuning runs applied the update: start again from the host tree
    plan.sync()
    ok, msg, _ = oracle.check_image(s, src.root, plan.image(), plan.device_base)
    assert ok, msg
    plan.relocate_update(op)
    plan.copy_back()
    plan.sync()
    cp = oracle.deep_copy(s, ref.root)
    oracle.update(s, cp.root, oop)
    oracle.copy_back(s, cp.root, ref.root, oop)
    ok, msg = oracle.trees_equal(s, src.root, ref.root)
    assert ok, msg
    plan.destroy()
