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
- Arrays past 2^32 elements: one struct holding x and y of 2^32 + 7 fp32
  (16 GiB each) through the staged deep copy, the update and the copy back,
  and through dc_roundtrip on a DC_PLAN_MAP_HOST plan; every element against
  the single-rounded x + 0.5*y.
"""
import ctypes
import functools

import numpy as np
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


BIG_N = (1 << 32) + 7  # fp32 elements per array: element indices pass 2^32, with a 3-element tail
BIG_CHUNK = 1 << 26


@functools.lru_cache(maxsize=2)
def big_base(which: int) -> np.ndarray:
    return np.random.default_rng(17 + which).random(BIG_CHUNK, dtype=np.float32) * 2 - 1


def big_shift(k: int, which: int) -> np.float32:
    return np.float32(k) / np.float32(64 << which)


def big_values(k: int, which: int, out=None) -> np.ndarray:
    """Chunk k of x (which = 0) or y (1): a seeded block in [-1, 1) shifted by
    a per-chunk constant, so that an element index that wrapped at 2^32 would
    read another chunk's values."""
    n = min(BIG_CHUNK, BIG_N - k * BIG_CHUNK)
    return np.add(big_base(which)[:n], big_shift(k, which), out=out if out is None else out[:n])


def big_chunks():
    return range((BIG_N + BIG_CHUNK - 1) // BIG_CHUNK)


def fill_big(a: np.ndarray, which: int):
    for k in big_chunks():
        big_values(k, which, out=a[k * BIG_CHUNK:(k + 1) * BIG_CHUNK])


def check_big(x: np.ndarray):
    w1, w2 = np.empty(BIG_CHUNK, np.float32), np.empty(BIG_CHUNK, np.float32)
    for k in big_chunks():
        got = x[k * BIG_CHUNK:(k + 1) * BIG_CHUNK]
        want = big_values(k, 0, out=w1)
        np.add(want, np.multiply(big_values(k, 1, out=w2), np.float32(0.5), out=w2[:got.size]),
               out=want)  # 0.5*y is exact: one rounding
        bad = np.flatnonzero(got.view(np.uint32) != want.view(np.uint32))
        assert bad.size == 0, (k, int(bad[0]) + k * BIG_CHUNK, float(got[bad[0]]), float(want[bad[0]]))


def host_available_bytes() -> int:
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    return 0


def test_arrays_past_2_32_elements():
    if host_available_bytes() < 110e9:
        pytest.skip("needs 110 GB of host memory (two 16 GiB arrays, a 32 GiB pinned arena)")
    torch.cuda.empty_cache()
    if torch.cuda.mem_get_info()[0] < (40 << 30):
        pytest.skip("needs 40 GiB of device memory")
    schema = tg.Schema([tg.Type("Big", 16, 8, [
        tg.Field("x", tg.ARRAY, 0, 4, count_const=BIG_N, elem_kind=tg.F32),
        tg.Field("y", tg.ARRAY, 8, 4, count_const=BIG_N, elem_kind=tg.F32)])])
    x = np.empty(BIG_N, dtype=np.float32)
    y = np.empty(BIG_N, dtype=np.float32)
    fill_big(y, 1)
    root = (ctypes.c_uint64 * 2)(x.ctypes.data, y.ctypes.data)
    op = dc.Op(x_field=0, y_field=1)
    for flags in (0, dc.PLAN_MAP_HOST):
        fill_big(x, 0)
        p = dc.Plan(schema, ctypes.addressof(root), flags=flags)
        assert p.info["nblocks"] == 3 and p.info["payload_bytes"] == 16 + 8 * BIG_N
        buf = p.bind()
        if flags == 0:  # the staged path: transfer + relocation, leaf update, copy back
            p.deep_copy()
            p.update(op)
            p.copy_back()
        else:  # the fused round trip: host x, y -> update -> arena and host
            p.roundtrip(op)
        # the device copy: both slots relocated, and x past element 2^32 updated
        ox, oy = p.blocks()[1]["offset"], p.blocks()[2]["offset"]
        slots = buf[:16].cpu().numpy().view(np.uint64)
        assert int(slots[0]) == buf.data_ptr() + ox and int(slots[1]) == buf.data_ptr() + oy
        xd = buf[ox:ox + 4 * BIG_N].view(torch.float32)
        for i in (0, (1 << 32) - 1, 1 << 32, BIG_N - 1):
            assert xd[i].item() == float(x[i]), (flags, i)
        check_big(x)
        for k in (0, BIG_N // BIG_CHUNK - 1, BIG_N // BIG_CHUNK):  # y is never written
            assert np.array_equal(y[k * BIG_CHUNK:(k + 1) * BIG_CHUNK], big_values(k, 1)), k
        del xd, buf
        p.destroy()
        torch.cuda.empty_cache()
