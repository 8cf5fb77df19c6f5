"""Parity of the CUDA path with the CPU oracle, element by element, through the
C ABI.  Copies, pointers and the fp32/fp64 updates must be bit-exact (0 ULP:
the kernels use __fadd_rn/__fmul_rn, one IEEE rounding per operation, as the
oracle does).  Covers the named workloads at full size (the sizes the
benchmark runs), small cases that span several tiles with ragged tails, the
paper's Linear/Dense/Listing-1 shapes, random schemas and the degenerate
cases (empty arrays, a lone struct, tiny segments)."""
import ctypes
import random

import numpy as np
import pytest
import torch

import oracle
import treegen as tg
from bump import BumpAllocator
import paper_1906_01128_b300 as dc

pytestmark = pytest.mark.gpu

NODE_LEAF = 4  # the node struct's child field


def ops_pair(kind=dc.OP_AXPY_HALF, sel=dc.SEL_ALL, type_=0, x=2, y=3, scale=1.0, path=()):
    return (dc.Op(kind, sel, type_, x, y, scale, list(path)),
            oracle.Op(kind, sel, type_, x, y, scale, list(path)))


PACK_BELOW = 64  # DC_PACK_BYTES: a packed plan's small arrays may start on their element alignment


def pack_of(plan):
    return PACK_BELOW if plan.flags & dc.PLAN_PACK_SMALL else 0


def image_ok(plan, schema, root_tree):
    ok, msg, seen = oracle.check_image(schema, root_tree, plan.image(), plan.device_base, pack_below=pack_of(plan))
    assert ok, msg
    return seen


def full_parity(make, op_kw=None, mode="leaf", verify=False, repeat=1, flags=0):
    """Deep copy `make()` with the CUDA path and the oracle, run the op
    `repeat` times on both, copy back on both, compare every stage."""
    src, ref = make(), make()
    s = src.schema
    plan = dc.Plan(s, src.root, flags=(dc.PLAN_VERIFY if verify else 0) | flags)
    plan.bind()
    plan.deep_copy()
    plan.sync()
    seen = image_ok(plan, s, src.root)
    c = oracle.count(s, src.root)
    assert (seen["nblocks"], seen["payload_bytes"], seen["nstructs"]) == (c["nblocks"], c["payload_bytes"],
                                                                         c["nstructs"])
    if op_kw is None:
        plan.copy_back(all_arrays=True)
        assert oracle.trees_equal(s, src.root, ref.root)[0]
        plan.destroy()
        return plan
    dop, oop = ops_pair(**op_kw)
    cp = oracle.deep_copy(s, ref.root)
    for _ in range(repeat):
        (plan.update if mode == "leaf" else plan.update_chase)(dop)
        oracle.update(s, cp.root, oop)
    plan.sync()
    image_ok(plan, s, cp.root)  # device arrays == the oracle's updated copy
    plan.copy_back()
    oracle.copy_back(s, cp.root, ref.root, oop)
    ok, msg = oracle.trees_equal(s, src.root, ref.root)
    assert ok, msg
    plan.destroy()
    src.free()
    ref.free()


# ---- named workloads at full size -------------------------------------------

def test_tiny_all_nodes():
    full_parity(lambda: tg.workload("tiny"), {})


def test_tiny_chain_to_last_level():
    full_parity(lambda: tg.workload("tiny"), dict(sel=dc.SEL_CHAIN, path=tg.leaf_path(4)))


def test_dense_all_nodes_full_size():
    full_parity(lambda: tg.workload("dense"), {}, verify=True)


def test_dense_all_nodes_mapped_host_pages():
    # array interiors moved straight from / to the caller's page-locked pages
    full_parity(lambda: tg.workload("dense"), {}, flags=dc.PLAN_MAP_HOST)
    full_parity(lambda: tg.workload("deep"), dict(sel=dc.SEL_CHAIN, path=tg.leaf_path(64)), flags=dc.PLAN_MAP_HOST)


@pytest.mark.parametrize("flags", [0, dc.PLAN_MAP_HOST])
def test_lengths_around_the_mapping_threshold(flags):
    # 16,000-17,000 fp32 per array: interiors of 0-2 pages above 64 KiB, heads and tails staged
    full_parity(lambda: tg.node_tree(3, 9, tg.uniform(16000, 17000), seed=31), None, flags=flags)
    full_parity(lambda: tg.node_tree(3, 9, tg.uniform(16000, 17000), seed=31), {}, flags=flags)
    full_parity(lambda: tg.node_tree(3, 9, tg.uniform(60000, 70000), seed=31), {}, flags=flags)


def test_mapped_pages_do_not_break_callers_copies():
    # while a MAP_HOST plan is bound, ordinary torch copies from other host memory work
    t = tg.workload("tiny")
    p = dc.Plan(t.schema, t.root, flags=dc.PLAN_MAP_HOST)
    p.bind()
    p.deep_copy()
    p.sync()
    for n in (1000, 100000, 3000000):
        x = torch.arange(n, dtype=torch.float32)
        assert torch.equal(x.cuda().cpu(), x)
    p.destroy()
    t.free()


def test_dense_chain_listing2_path():
    full_parity(lambda: tg.workload("dense"), dict(sel=dc.SEL_CHAIN, path=[(NODE_LEAF, 15), (NODE_LEAF, 15)]))


def test_deep_chain_to_leaf_full_size():
    full_parity(lambda: tg.workload("deep"), dict(sel=dc.SEL_CHAIN, path=tg.leaf_path(64)))


@pytest.mark.parametrize("case", ["dense", "deep_chain", "reloc_stress", "linear_scale_f64", "ragged"])
def test_direct_load_leaf_kernel(case, monkeypatch):
    """DC_LEAF_TMA=0 selects the direct-load leaf kernel instead of the default
    bulk-copy one; its results are the oracle's too."""
    monkeypatch.setenv("DC_LEAF_TMA", "0")
    make, op = {
        "dense": (lambda: tg.workload("dense"), {}),
        "deep_chain": (lambda: tg.workload("deep"), dict(sel=dc.SEL_CHAIN, path=tg.leaf_path(64))),
        "reloc_stress": (lambda: tg.workload("reloc_stress"), {}),
        "linear_scale_f64": (lambda: tg.linear_tree(6, 100001, "allinit", seed=3), dict(kind=dc.OP_SCALE, x=2, scale=1.5)),
        "ragged": (lambda: tg.node_tree(4, 6, tg.uniform(0, 3000), seed=8), {}),
    }[case]
    full_parity(make, op, repeat=2)


def test_device_scan_relocation():
    """DC_PLAN_DEVICE_SCAN: the relocation derives the offsets from the targets'
    sizes with segmented warp-shuffle prefix sums; the device image and the results are
    the oracle's, as with the default offset records (dense: two tiles; a
    ragged tree of ~13,000 blocks: 18 tiles and lane groups of uneven runs)."""
    full_parity(lambda: tg.workload("dense"), {}, flags=dc.PLAN_DEVICE_SCAN)
    full_parity(lambda: tg.node_tree(4, 16, tg.uniform(1, 40), seed=21), {}, verify=True,
                flags=dc.PLAN_DEVICE_SCAN)


def test_device_scan_random_schemas():
    """Scan records on random schemas (several array and child lanes per struct):
    lane groups start at every position of a 32-record slice, so the warp scans'
    segments begin mid-slice; the device-side slot check compares every offset."""
    rng = random.Random(5151)
    for i in range(40):
        schema, levels, rules = tg.random_schema(rng)
        full_parity(lambda: tg.Tree(schema, levels, rules, seed=900 + i), None, verify=True,
                    flags=dc.PLAN_DEVICE_SCAN)


@pytest.mark.parametrize("threads", [128, 256, 512])
def test_device_scan_fused_launch_each_cta_size(threads):
    # the scan form inside the persistent launch: 4, 8 and 16 warps share a tile's slices
    src, ref = tg.node_tree(4, 16, tg.uniform(1, 40), seed=21), tg.node_tree(4, 16, tg.uniform(1, 40), seed=21)
    s = src.schema
    plan = dc.Plan(s, src.root, flags=dc.PLAN_DEVICE_SCAN)
    plan.bind()
    dop, oop = ops_pair()
    cp = oracle.deep_copy(s, ref.root)
    plan.deep_copy()
    plan.set_split(dop, threads, 2)
    for _ in range(2):  # each launch relocates again and updates once more
        plan.relocate_update(dop)
        plan.sync()
        oracle.update(s, cp.root, oop)
        image_ok(plan, s, cp.root)
    plan.destroy()
    src.free()
    ref.free()


def test_reloc_stress_device_scan():
    # the 2.3M-slot tree through the scan form, with the device-side slot check on
    full_parity(lambda: tg.workload("reloc_stress"), {}, verify=True, flags=dc.PLAN_DEVICE_SCAN)


def test_reloc_stress_many_tiles():
    # 1,118,481 nodes, 2,306,868 blocks: 4,370 relocation tiles over the 35.8 MB struct lane,
    # several per CTA through the two-stage pipeline, with the device-side slot check on
    full_parity(lambda: tg.workload("reloc_stress"), {}, verify=True)


# ---- comparison paths --------------------------------------------------------

def test_chase_matches_oracle_dense_all():
    full_parity(lambda: tg.workload("dense"), {}, mode="chase")


def test_chase_matches_oracle_deep_chain():
    full_parity(lambda: tg.node_tree(64, 1, 1024, 1 << 18, seed=3), dict(sel=dc.SEL_CHAIN, path=tg.leaf_path(64)),
                mode="chase")


@pytest.mark.parametrize("prefetch", [False, True])
def test_uvm_matches_oracle(prefetch):
    src = tg.node_tree(3, 16, tg.lognormal(4096, 1.2, 65536), seed=2)
    ref = tg.node_tree(3, 16, tg.lognormal(4096, 1.2, 65536), seed=2)
    s = src.schema
    u = dc.Uvm(s, src.root)
    if prefetch:
        u.prefetch(True)
    dop, oop = ops_pair()
    u.update(dop)
    u.sync()
    cp = oracle.deep_copy(s, ref.root)
    oracle.update(s, cp.root, oop)
    ok, msg = oracle.trees_equal(s, u.root, cp.root)  # the managed tree itself
    assert ok, msg
    u.copy_back()
    oracle.copy_back(s, cp.root, ref.root, oop)
    assert oracle.trees_equal(s, src.root, ref.root)[0]
    u.destroy()


def test_uvm_chain_scale_f64_linear():
    src, ref = tg.linear_tree(8, 5000, "llinit", seed=8), tg.linear_tree(8, 5000, "llinit", seed=8)
    s = src.schema
    u = dc.Uvm(s, src.root)
    kw = dict(kind=dc.OP_SCALE, sel=dc.SEL_CHAIN, x=2, scale=1.5, path=[(3, 0)] * 7)
    dop, oop = ops_pair(**kw)
    u.update(dop)
    u.sync()
    u.copy_back()
    cp = oracle.deep_copy(s, ref.root)
    oracle.update(s, cp.root, oop)
    oracle.copy_back(s, cp.root, ref.root, oop)
    assert oracle.trees_equal(s, src.root, ref.root)[0]
    u.destroy()


# ---- the paper's shapes --------------------------------------------------------

@pytest.mark.parametrize("layout", ["allinit", "llinit"])
def test_linear_scale_f64(layout):
    kw = dict(kind=dc.OP_SCALE, x=2, scale=1.5)
    if layout == "llinit":
        kw.update(sel=dc.SEL_CHAIN, path=[(3, 0)] * 9)
    full_parity(lambda: tg.linear_tree(10, 10 ** 5, layout, seed=10), kw)


def test_dense_listing2_chain_scale():
    q, D = 8, 3
    full_parity(lambda: tg.dense_tree(q, 1000, D, seed=4),
                dict(kind=dc.OP_SCALE, sel=dc.SEL_CHAIN, type_=D, x=1, scale=1.25, path=[(3, q - 1)] * D))
    full_parity(lambda: tg.dense_tree(q, 1000, D, seed=4),
                dict(kind=dc.OP_SCALE, sel=dc.SEL_CHAIN, type_=D, x=1, scale=1.25, path=[(3, q - 1)] * D),
                mode="chase")


def test_dense_paper_all_levels_scale_f64():
    # the Dense struct has one array per level: scale every level's A, level type by type
    for lvl in range(4):
        full_parity(lambda: tg.dense_tree(4, 300, 3, seed=5),
                    dict(kind=dc.OP_SCALE, type_=lvl, x=2 if lvl < 3 else 1, scale=0.75))


def test_listing1_chain():
    full_parity(lambda: tg.listing1_tree(100000, seed=1),
                dict(kind=dc.OP_SCALE, sel=dc.SEL_CHAIN, type_=2, x=1, scale=3.0, path=[(1, 0), (1, 0)]))


# ---- ragged and degenerate cases -------------------------------------------------

def test_ragged_lengths_and_empty_nodes():
    full_parity(lambda: tg.node_tree(3, 7, tg.uniform(0, 3000), seed=12), {})
    full_parity(lambda: tg.node_tree(3, 7, tg.uniform(0, 3000), seed=12), {}, mode="chase")


def test_many_tiny_segments():
    # 22,621 nodes of 1-9 elements: many segments per tile, multi-tile relocation
    full_parity(lambda: tg.node_tree(5, 12, tg.uniform(1, 9), seed=13), {}, verify=True)
    full_parity(lambda: tg.node_tree(5, 12, tg.uniform(1, 9), seed=13), {}, mode="chase")


class CNode(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nchild", ctypes.c_int32), ("position", ctypes.c_void_p),
                ("velocity", ctypes.c_void_p), ("child", ctypes.c_void_p)]


class HandTree:
    """root {n = 0 but position/velocity set to junk} -> 3 children with data:
    the root's slots must come out NULL; its block takes the staged path while
    the others move through mapped host pages."""

    def __init__(self):
        self.schema = tg.node_schema()
        self.junk = (ctypes.c_float * 4)()
        self.arrs = [(ctypes.c_float * 1000)(*[float(i % 97) / 128 for i in range(1000)]) for _ in range(6)]
        self.kids = (CNode * 3)()
        for j in range(3):
            self.kids[j] = CNode(1000 - j, 0, ctypes.addressof(self.arrs[2 * j]), ctypes.addressof(self.arrs[2 * j + 1]),
                                 None)
        self.node = CNode(0, 3, ctypes.addressof(self.junk), ctypes.addressof(self.junk), ctypes.addressof(self.kids))
        self.root = ctypes.addressof(self.node)

    def free(self):
        pass


@pytest.mark.parametrize("flags", [0, dc.PLAN_MAP_HOST])
def test_count_zero_slot_is_nulled_on_the_device(flags):
    full_parity(HandTree, {}, flags=flags)
    full_parity(HandTree, None, flags=flags)


def test_lone_struct_and_empty_tree():
    full_parity(lambda: tg.node_tree(1, 0, 0, seed=1), None)
    full_parity(lambda: tg.node_tree(1, 0, 5, seed=1), {})
    full_parity(lambda: tg.node_tree(4, 2, 0, seed=1), {})  # structs only, no arrays


def test_repeated_updates_reuse_the_table():
    full_parity(lambda: tg.node_tree(3, 5, tg.uniform(1, 999), seed=14), {}, repeat=3)
    full_parity(lambda: tg.node_tree(3, 5, tg.uniform(1, 999), seed=14),
                dict(kind=dc.OP_SCALE, scale=-2.0), repeat=2)


def test_random_schemas_deep_copy_and_copy_back():
    rng = random.Random(4242)
    for i in range(80):
        schema, levels, rules = tg.random_schema(rng)
        full_parity(lambda: tg.Tree(schema, levels, rules, seed=500 + i), None)


# ---- re-copy, resolution, relocation check ---------------------------------------

def test_second_deep_copy_restores_the_image():
    t = tg.node_tree(4, 6, tg.uniform(0, 700), seed=15)
    p = dc.Plan(t.schema, t.root, flags=dc.PLAN_VERIFY)
    p.bind()
    p.deep_copy()
    p.sync()
    first = p.image().copy()
    p.update(dc.Op())
    p.deep_copy()
    p.deep_copy()
    p.sync()
    assert np.array_equal(first, p.image())
    p.destroy()


def test_resolve_chain_matches_device_walk_and_oracle():
    t = tg.workload("dense")
    p = dc.Plan(t.schema, t.root)
    p.bind()
    p.deep_copy()
    p.sync()
    image_ok(p, t.schema, t.root)  # the walk below dereferences relocated pointers
    img, base = p.image(), p.device_base
    rng = random.Random(3)
    paths = [[], [(NODE_LEAF, 15)], [(NODE_LEAF, 15), (NODE_LEAF, 15)], [(NODE_LEAF, 3), (NODE_LEAF, 7), (2, 0)]]
    for _ in range(40):
        path = [(NODE_LEAF, rng.randrange(16)) for _ in range(rng.randint(0, 2))]
        path.append((rng.choice([2, 3]), 0))
        paths.append(path)
    for path in paths:
        a = p.resolve(path)
        assert a == p.verify_chain(path) == oracle.image_resolve(t.schema, img, base, path)
    deep = tg.workload("deep")
    q = dc.Plan(deep.schema, deep.root)
    q.bind()
    q.deep_copy()
    q.sync()
    image_ok(q, deep.schema, deep.root)
    path = tg.leaf_path(64) + [(2, (1 << 26) - 1)]
    assert q.resolve(path) == q.verify_chain(path) == oracle.image_resolve(deep.schema, q.image(), q.device_base, path)
    p.destroy()
    q.destroy()


def test_kernels_are_launched_by_the_library():
    n0 = dc.kernel_launches()
    full_parity(lambda: tg.node_tree(2, 3, 100, seed=1), {})
    assert dc.kernel_launches() >= n0 + 2


def test_stream_ordering_on_a_side_stream():
    src, ref = tg.workload("tiny"), tg.workload("tiny")
    s = src.schema
    st = torch.cuda.Stream()
    p = dc.Plan(s, src.root)
    p.bind(stream=st)
    with torch.cuda.stream(st):
        p.deep_copy(stream=st)
        p.update(dc.Op(), stream=st)
        p.copy_back(stream=st)
    cp = oracle.deep_copy(s, ref.root)
    oracle.update(s, cp.root, oracle.Op())
    oracle.copy_back(s, cp.root, ref.root, oracle.Op())
    assert oracle.trees_equal(s, src.root, ref.root)[0]
    p.destroy()


# ---- the fused round trip (deep copy + update + copy back in one call) ------------------

def step_parity(make, op_kw, flags, repeat=1):
    src, ref = make(), make()
    s = src.schema
    plan = dc.Plan(s, src.root, flags=flags)
    plan.bind()
    dop, oop = ops_pair(**op_kw)
    for _ in range(repeat):
        plan.roundtrip(dop)
        cp = oracle.deep_copy(s, ref.root)  # the oracle's pass: copy, update, copy back
        oracle.update(s, cp.root, oop)
        oracle.copy_back(s, cp.root, ref.root, oop)
        image_ok(plan, s, cp.root)  # the arena holds the updated copy
        ok, msg = oracle.trees_equal(s, src.root, ref.root)
        assert ok, msg
    plan.destroy()
    src.free()
    ref.free()


@pytest.mark.parametrize("flags", [dc.PLAN_MAP_HOST, 0])
def test_step_dense_all_nodes(flags):
    step_parity(lambda: tg.workload("dense"), {}, flags, repeat=2)


def test_step_deep_chain_and_ragged():
    step_parity(lambda: tg.workload("deep"), dict(sel=dc.SEL_CHAIN, path=tg.leaf_path(64)), dc.PLAN_MAP_HOST)
    step_parity(lambda: tg.node_tree(3, 9, tg.uniform(0, 40000), seed=41), {}, dc.PLAN_MAP_HOST, repeat=2)
    step_parity(lambda: tg.node_tree(5, 12, tg.uniform(1, 9), seed=13), {}, dc.PLAN_MAP_HOST)


def test_step_scale_f64_and_null_slots():
    step_parity(lambda: tg.linear_tree(6, 100000, "allinit", seed=3), dict(kind=dc.OP_SCALE, x=2, scale=1.5),
                dc.PLAN_MAP_HOST)
    step_parity(HandTree, {}, dc.PLAN_MAP_HOST, repeat=2)


# ---- forests: one plan for many trees; fused relocation + update -------------------

def forest_parity(ntrees, t_max, mode, flags=0, seed=4):
    src = tg.batched(ntrees, seed=seed, t_max=t_max)
    ref = tg.batched(ntrees, seed=seed, t_max=t_max)
    s = src[0].schema
    plan = dc.Plan(s, [t.root for t in src], flags=flags)
    info = plan.info
    assert info["ntrees"] == ntrees
    plan.bind()
    dop, oop = ops_pair()
    if mode == "roundtrip":
        plan.roundtrip(dop)
    else:
        plan.deep_copy()
        plan.sync()
        img, base = plan.image(), plan.device_base
        for i, t in enumerate(src):  # every tree of the arena is its source's replica
            ok, msg, _ = oracle.check_image(s, t.root, img, base, plan.root_offset(i), pack_below=pack_of(plan))
            assert ok, (i, msg)
        if mode == "fused":
            plan.relocate_update(dop)
        elif mode == "tuned":
            plan.autotune(dop)
            plan.deep_copy()  # the tuning runs applied the update: start again
            plan.relocate_update(dop)
        elif mode.startswith("split"):  # a pinned launch shape: "split-THREADS-CTAS"
            _, threads, ctas = mode.split("-")
            plan.set_split(dop, int(threads), int(ctas))
            plan.relocate_update(dop)
        elif mode == "graph":
            plan.relocate_update(dop)  # puts the op's tables on the device
            plan.sync()
            plan.deep_copy()
            g = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                with torch.cuda.graph(g, stream=side):
                    plan.relocate_update(dop, stream=side)
            torch.cuda.current_stream().wait_stream(side)
            plan.deep_copy()  # capture does not run the kernel; start from the copy
            plan.sync()
            g.replay()
        else:
            plan.update(dop)
        plan.copy_back()
    for t, r in zip(src, ref):
        cp = oracle.deep_copy(s, r.root)
        oracle.update(s, cp.root, oop)
        oracle.copy_back(s, cp.root, r.root, oop)
        ok, msg = oracle.trees_equal(s, t.root, r.root)
        assert ok, msg
    plan.destroy()


@pytest.mark.parametrize("mode", ["plain", "fused", "tuned", "split-128-1", "split-512-64", "graph", "roundtrip"])
def test_forest_of_uneven_trees(mode):
    forest_parity(300, 256 << 10, mode, flags=dc.PLAN_MAP_HOST if mode == "roundtrip" else 0)


@pytest.mark.parametrize("mode", ["fused", "split-128-1"])
def test_forest_fused_launch_with_device_scan(mode):
    # the persistent relocation + update launch with scan records
    forest_parity(300, 256 << 10, mode, flags=dc.PLAN_DEVICE_SCAN)


def test_forest_resolution_per_tree():
    trees = tg.batched(20, seed=9, t_max=64 << 10)
    s = trees[0].schema
    p = dc.Plan(s, [t.root for t in trees])
    p.bind()
    p.deep_copy()
    p.sync()
    img, base = p.image(), p.device_base
    for i, t in enumerate(trees):
        ok, msg, _ = oracle.check_image(s, t.root, img, base, p.root_offset(i))
        assert ok, msg
        assert p.resolve_in(i, []) == base + p.root_offset(i)
        assert p.resolve_in(i, [(2, 0)]) == oracle.image_resolve(s, img, base, [(2, 0)], p.root_offset(i))
    p.destroy()


def test_fused_single_tree_workloads():
    full_parity(lambda: tg.workload("dense"), {}, mode="leaf")
    for make in (lambda: tg.workload("dense"), lambda: tg.node_tree(5, 12, tg.uniform(1, 9), seed=13)):
        src, ref = make(), make()
        s = src.schema
        plan = dc.Plan(s, src.root)
        plan.bind()
        plan.deep_copy()
        dop, oop = ops_pair()
        plan.relocate_update(dop)
        plan.sync()
        cp = oracle.deep_copy(s, ref.root)
        oracle.update(s, cp.root, oop)
        image_ok(plan, s, cp.root)
        plan.destroy()


def node64_tree(levels, fanout, n, seed):
    """The node struct with fp64 position and velocity arrays (an AXPY in fp64
    needs two arrays of one struct)."""
    sch = tg.node_schema()
    for f in sch.types[0].fields[2:4]:
        f.elem_size, f.elem_kind = 8, tg.F64
    rules = [tg.Rule(0, 0, n if isinstance(n, tuple) else tg.const(n), n if isinstance(n, tuple) else tg.const(n)),
             tg.Rule(0, 1, tg.const(fanout), tg.const(0))]
    return tg.Tree(sch, levels, rules, seed, name=f"node64-{levels}-{fanout}")


# fp64 x += 0.5*y, and fp32 x *= scale with scales that are not fp32 numbers
# (the kernel must multiply by the scale rounded to float, once)
ROUNDING_CASES = {
    "node64_axpy": (lambda: node64_tree(3, 7, tg.uniform(0, 5000), seed=31), {}),
    "node64_chain_axpy": (lambda: node64_tree(3, 7, tg.uniform(1, 5000), seed=32),
                          dict(sel=dc.SEL_CHAIN, path=[(NODE_LEAF, 3), (NODE_LEAF, 1)])),
    "listing1_axpy_f64": (lambda: tg.listing1_tree(100003, seed=33), dict(type_=2, x=1, y=2)),
    "node_scale_f32_inexact": (lambda: tg.node_tree(3, 7, tg.uniform(0, 5000), seed=34),
                               dict(kind=dc.OP_SCALE, scale=1.1)),
    "node_chain_scale_f32_inexact": (lambda: tg.node_tree(3, 7, tg.uniform(1, 5000), seed=35),
                                     dict(kind=dc.OP_SCALE, sel=dc.SEL_CHAIN, scale=-0.7,
                                          path=[(NODE_LEAF, 6), (NODE_LEAF, 0)])),
}


@pytest.mark.parametrize("case", sorted(ROUNDING_CASES))
def test_axpy_f64_and_inexact_f32_scale(case, monkeypatch):
    """Every path that runs the update, against the oracle at 0 ULP: the
    bulk-copy leaf kernel (dc_update_leaves, twice), the direct-load one, the
    pointer chase, and the one-call round trip (dc_roundtrip) on mapped and
    staged plans.  dc_relocate_update takes the same cases in
    test_fused_launch_every_kind_and_width."""
    make, kw = ROUNDING_CASES[case]
    full_parity(make, kw, repeat=2)
    full_parity(make, kw, mode="chase")
    step_parity(make, kw, dc.PLAN_MAP_HOST, repeat=2)
    step_parity(make, kw, 0)
    monkeypatch.setenv("DC_LEAF_TMA", "0")
    full_parity(make, kw)


def test_axpy_f64_dense_shape_full_size():
    # the dense workload's shape and lengths (3 levels, fanout 16, lognormal
    # median 65,536) with fp64 arrays: 677 MB, through the leaf update, the
    # persistent fused launch and the round trip
    make = lambda: node64_tree(3, 16, tg.lognormal(65536, 1.2, 4194304), seed=2)
    full_parity(make, {})
    step_parity(make, {}, dc.PLAN_MAP_HOST)
    src, ref = make(), make()
    s = src.schema
    plan = dc.Plan(s, src.root)
    plan.bind()
    plan.deep_copy()
    dop, oop = ops_pair()
    plan.relocate_update(dop)
    plan.sync()
    cp = oracle.deep_copy(s, ref.root)
    oracle.update(s, cp.root, oop)
    image_ok(plan, s, cp.root)
    plan.destroy()


FUSED_CASES = {
    **ROUNDING_CASES,
    # Linear chain, fp64 A: x *= 1.5 on every level (the paper's kernel)
    "linear_scale_f64": (lambda: tg.linear_tree(6, 100000, "allinit", seed=3), dict(kind=dc.OP_SCALE, x=2, scale=1.5)),
    # the same on the last level only, reached by a chain
    "linear_chain_f64": (lambda: tg.linear_tree(8, 70001, "allinit", seed=4),
                         dict(kind=dc.OP_SCALE, sel=dc.SEL_CHAIN, x=2, scale=-0.75, path=[(3, 0)] * 7)),
    # node tree, fp32: x *= scale, and x += 0.5*y on one node's chain
    "node_scale_f32": (lambda: tg.node_tree(4, 6, tg.uniform(0, 3000), seed=8), dict(kind=dc.OP_SCALE, scale=3.0)),
    "node_chain_axpy": (lambda: tg.node_tree(4, 6, tg.uniform(1, 3000), seed=9),
                        dict(sel=dc.SEL_CHAIN, path=[(NODE_LEAF, 5), (NODE_LEAF, 2)])),
}


@pytest.mark.parametrize("threads", [128, 256, 512])
@pytest.mark.parametrize("case", sorted(FUSED_CASES))
def test_fused_launch_every_kind_and_width(case, threads):
    """dc_relocate_update's instances beyond fp32 x += 0.5*y over every node:
    fp64 and fp32 SCALE, chain selections, at each CTA size (pinned with
    dc_set_split), twice in a row: the device image after each launch equals
    the oracle's copy updated as many times."""
    make, op_kw = FUSED_CASES[case]
    src, ref = make(), make()
    s = src.schema
    plan = dc.Plan(s, src.root)
    plan.bind()
    plan.deep_copy()
    dop, oop = ops_pair(**op_kw)
    plan.set_split(dop, threads, 2)
    cp = oracle.deep_copy(s, ref.root)
    for _ in range(2):
        plan.relocate_update(dop)
        plan.sync()
        oracle.update(s, cp.root, oop)
        image_ok(plan, s, cp.root)
    plan.destroy()
    src.free()
    ref.free()


# ---- host arenas (allocation requests served from one pinned buffer) -----------------

def arena_case(make_tree, op_kw, mode, arena_bytes, flags=0):
    arena = dc.HostArena(arena_bytes)
    src = make_tree(arena.allocator)  # every block of the source tree comes from the arena
    ref = make_tree(None)
    assert arena.used >= src.payload_bytes
    s = src.schema
    plan = dc.Plan(s, src.root, flags=flags)
    plan.bind()
    dop, oop = ops_pair(**op_kw)
    if mode == "calls":
        plan.deep_copy()
        plan.sync()
        image_ok(plan, s, src.root)
        plan.update(dop)
        plan.copy_back()
    elif mode == "roundtrip":
        plan.roundtrip(dop)
    else:
        plan.roundtrip_selected(dop)
    cp = oracle.deep_copy(s, ref.root)
    oracle.update(s, cp.root, oop)
    oracle.copy_back(s, cp.root, ref.root, oop)
    ok, msg = oracle.trees_equal(s, src.root, ref.root)
    assert ok, msg
    plan.destroy()
    src.free()
    arena.destroy()


@pytest.mark.parametrize("mode", ["calls", "roundtrip", "selected"])
def test_trees_built_in_a_host_arena(mode):
    arena_case(lambda a: tg.workload("dense", alloc=a), {}, mode, 400 << 20)
    arena_case(lambda a: tg.node_tree(5, 12, tg.uniform(1, 9), seed=13, alloc=a), {}, mode, 64 << 20)
    arena_case(lambda a: tg.node_tree(64, 1, 1024, 1 << 20, seed=3, alloc=a),
               dict(sel=dc.SEL_CHAIN, path=tg.leaf_path(64)), mode, 64 << 20)
    # host-arena blocks move in place: with DC_PLAN_SPANS nothing is left to stage
    arena_case(lambda a: tg.node_tree(5, 12, tg.uniform(1, 9), seed=13, alloc=a), {}, mode, 64 << 20,
               flags=dc.PLAN_SPANS)


# ---- span staging: host spans copied whole, every block placed by one device launch ----

SPAN_CASES = {
    "ragged": (lambda: tg.node_tree(4, 6, tg.uniform(0, 3000), seed=8), {}),
    "small_arrays": (lambda: tg.node_tree(5, 8, tg.uniform(1, 30), seed=41), {}),
    "listing1_f64": (lambda: tg.listing1_tree(3001, seed=33), dict(type_=2, x=1, y=2)),
    "deep_chain": (lambda: tg.node_tree(64, 1, 1024, 1 << 18, seed=3), dict(sel=dc.SEL_CHAIN, path=tg.leaf_path(64))),
}


@pytest.mark.parametrize("case", sorted(SPAN_CASES))
def test_span_staging(case):
    """DC_PLAN_SPANS on trees the rule would stage block by block: the device image, the
    updates and the copy back equal the oracle's, with the slot check, on a packed plan
    and with the device scan."""
    make, kw = SPAN_CASES[case]
    t = make()
    p = dc.Plan(t.schema, t.root, flags=dc.PLAN_SPANS)
    assert p.info["staging_bytes"] >= t.payload_bytes  # the spans hold every staged block
    p.destroy()
    t.free()
    full_parity(make, kw, flags=dc.PLAN_SPANS, verify=True, repeat=2)
    full_parity(make, None, flags=dc.PLAN_SPANS)
    full_parity(make, kw, flags=dc.PLAN_SPANS | dc.PLAN_PACK_SMALL, verify=True)
    full_parity(make, kw, flags=dc.PLAN_SPANS | dc.PLAN_DEVICE_SCAN)


@pytest.mark.parametrize("flags", [0, dc.PLAN_PACK_SMALL])
def test_span_placement_zeroes_the_slots_padding(flags):
    """The placement writes each block and then zeros up to its 16-byte slot end (or the
    next block), so after a deep copy by spans every byte of the data region outside the
    blocks is zero, whatever the buffer held before; the blocks equal the oracle's."""
    for make, _ in SPAN_CASES.values():
        t = make()
        plan = dc.Plan(t.schema, t.root, flags=dc.PLAN_SPANS | flags)
        buf = plan.bind()
        n = plan.info["data_bytes"]
        buf[:n].fill_(0xAB)
        plan.deep_copy()
        plan.sync()
        image_ok(plan, t.schema, t.root)
        img = plan.image()[:n].copy()
        for b in plan.blocks():
            img[b["offset"]:b["offset"] + b["bytes"]] = 0
        assert not img.any(), int(np.flatnonzero(img)[0])
        plan.destroy()
        t.free()


@pytest.mark.parametrize("min_align", [8])
def test_span_staging_of_blocks_off_16_byte_boundaries(min_align):
    """Host blocks at 8-byte aligned addresses (a packing allocator's): the staging area
    keeps each span's phase, so the placement reads off 16 bytes and takes its 8-, 4- and 1-byte
    steps, for small pieces (one lane) and large ones (a warp)."""
    for make_kw in (dict(levels=4, fanout=8, length=10), dict(levels=3, fanout=6, length=tg.uniform(1, 3000))):
        def make(alloc=None):
            return tg.node_tree(make_kw["levels"], make_kw["fanout"], make_kw["length"], seed=77, alloc=alloc)
        bump = BumpAllocator(64 << 20, gap=4, min_align=min_align)
        src, ref = make(bump.alloc), make()
        s = src.schema
        assert any(a % 16 for a, _ in bump.blocks)
        for flags in (dc.PLAN_SPANS, dc.PLAN_SPANS | dc.PLAN_PACK_SMALL):
            plan = dc.Plan(s, src.root, flags=flags | dc.PLAN_VERIFY)
            plan.bind()
            plan.deep_copy()
            plan.sync()
            image_ok(plan, s, src.root)
            dop, oop = ops_pair()
            plan.update(dop)
            plan.copy_back()
            cp = oracle.deep_copy(s, ref.root)
            oracle.update(s, cp.root, oop)
            oracle.copy_back(s, cp.root, ref.root, oop)
            ok, msg = oracle.trees_equal(s, src.root, ref.root)
            assert ok, msg
            plan.destroy()
        src.free()
        ref.free()


def test_span_staging_with_part_of_the_tree_in_a_host_arena():
    """Every other block from a library host arena (moved in place, never staged) and the rest
    from one bump buffer (staged by host spans): the placement table skips the arena's blocks and
    the image, the update and the copy back equal the oracle's, with spans forced and by default."""
    from bump import ALLOC_FN
    for flags in (dc.PLAN_SPANS, 0):
        arena = dc.HostArena(64 << 20)
        bump = BumpAllocator(64 << 20)
        turn = [0]

        def alternate(ctx, nbytes, align):
            turn[0] += 1
            return arena.alloc(nbytes, max(align, 16)) if turn[0] % 2 else bump._alloc(None, nbytes, align)

        fn = ALLOC_FN(alternate)
        mk = lambda alloc=None: tg.node_tree(4, 8, tg.uniform(1, 300), seed=91, alloc=alloc)  # noqa: E731
        src, ref = mk((ctypes.cast(fn, ctypes.c_void_p).value, None)), mk()
        s = src.schema
        assert arena.used > 0 and bump.blocks
        plan = dc.Plan(s, src.root, flags=flags | dc.PLAN_VERIFY)
        if flags:
            assert plan.info["staging_bytes"] > 0
        plan.bind()
        plan.deep_copy()
        plan.sync()
        image_ok(plan, s, src.root)
        dop, oop = ops_pair()
        plan.update(dop)
        plan.copy_back()
        cp = oracle.deep_copy(s, ref.root)
        oracle.update(s, cp.root, oop)
        oracle.copy_back(s, cp.root, ref.root, oop)
        ok, msg = oracle.trees_equal(s, src.root, ref.root)
        assert ok, msg
        plan.destroy()
        src.free()
        ref.free()
        arena.destroy()


def test_span_staging_null_slots_and_random_schemas():
    # count-0 slots with a non-NULL host value are zeroed in the staging area
    full_parity(HandTree, {}, flags=dc.PLAN_SPANS)
    full_parity(HandTree, None, flags=dc.PLAN_SPANS)
    # a forest of 300 uneven trees: their spans, then one persistent relocation + update launch
    forest_parity(300, 256 << 10, "fused", flags=dc.PLAN_SPANS)
    rng = random.Random(6161)
    for i in range(40):
        schema, levels, rules = tg.random_schema(rng)
        full_parity(lambda: tg.Tree(schema, levels, rules, seed=1100 + i), None, flags=dc.PLAN_SPANS, verify=True)


def test_span_staging_by_the_rule_on_the_pointer_heavy_tree(monkeypatch):
    """The 1.1M-node tree of 40-byte arrays stages by spans on the default plan: repeated
    deep copies, the update, the copy back, the round trip, the selected-arrays round trip
    and a selective deep copy on one plan; with DC_SPANS=0 the same tree stages block by
    block."""
    bump = BumpAllocator(200 << 20)  # a compact host layout, whatever the process heap looks like
    src, ref = tg.workload("reloc_stress", alloc=bump.alloc), tg.workload("reloc_stress")
    s = src.schema
    plan = dc.Plan(s, src.root)
    assert plan.info["staging_bytes"] > 0
    plan.bind()
    dop, oop = ops_pair()
    cp = oracle.deep_copy(s, ref.root)
    for _ in range(2):
        plan.deep_copy()
        plan.sync()
        image_ok(plan, s, src.root)
    plan.update(dop)
    oracle.update(s, cp.root, oop)
    plan.copy_back()
    oracle.copy_back(s, cp.root, ref.root, oop)
    assert oracle.trees_equal(s, src.root, ref.root)[0]
    plan.roundtrip(dop)  # deep copy + update + copy back, from the updated host tree
    oracle.update(s, cp.root, oop)
    oracle.copy_back(s, cp.root, ref.root, oop)
    assert oracle.trees_equal(s, src.root, ref.root)[0]
    plan.roundtrip_selected(dop)  # only the op's arrays, through the pinned arena at their arena offsets
    oracle.update(s, cp.root, oop)
    oracle.copy_back(s, cp.root, ref.root, oop)
    assert oracle.trees_equal(s, src.root, ref.root)[0]
    path = tg.leaf_path(6)
    dchain, _ = ops_pair(sel=dc.SEL_CHAIN, path=path)
    plan.deep_copy_selected(dchain)  # block by block, into the same pinned arena
    plan.sync()
    ok, msg = oracle.check_chain_image(s, src.root, plan.image(), plan.device_base, path, 2, 3)
    assert ok, msg
    plan.destroy()
    src.free()
    ref.free()
    del bump
    monkeypatch.setenv("DC_SPANS", "0")
    t = tg.workload("reloc_stress")
    p = dc.Plan(t.schema, t.root)
    assert p.info["staging_bytes"] == 0
    p.destroy()
    t.free()
    full_parity(lambda: tg.workload("reloc_stress"), {}, verify=True)


# ---- the pointerchain transfer scheme: only the op's arrays move ----------------------

@pytest.mark.parametrize("flags", [0, dc.PLAN_MAP_HOST])
def test_roundtrip_selected_matches_the_oracle(flags):
    cases = [
        (lambda: tg.workload("deep"), dict(sel=dc.SEL_CHAIN, path=tg.leaf_path(64))),
        (lambda: tg.workload("dense"), {}),
        (lambda: tg.workload("dense"), dict(sel=dc.SEL_CHAIN, path=[(NODE_LEAF, 15), (NODE_LEAF, 15)])),
        (lambda: tg.linear_tree(10, 10 ** 6, "allinit", seed=8),
         dict(kind=dc.OP_SCALE, sel=dc.SEL_CHAIN, x=2, scale=1.5, path=[(3, 0)] * 9)),
    ]
    for make, kw in cases:
        src, ref = make(), make()
        s = src.schema
        plan = dc.Plan(s, src.root, flags=flags)
        plan.bind()
        dop, oop = ops_pair(**kw)
        for _ in range(2):
            plan.roundtrip_selected(dop)
            cp = oracle.deep_copy(s, ref.root)
            oracle.update(s, cp.root, oop)
            oracle.copy_back(s, cp.root, ref.root, oop)
            ok, msg = oracle.trees_equal(s, src.root, ref.root)
            assert ok, msg
        plan.destroy()
        src.free()
        ref.free()


# ---- the selective deep copy of a chain (Sec. 2; Sec. 4.1.2's LLused layouts) ----------

SELECTIVE_CASES = {
    # Linear allinit-LLused: every level has its A, the kernel scales the last level's
    "linear_allinit_llused": (lambda: tg.linear_tree(10, 10 ** 5, "allinit", seed=8),
                              dict(kind=dc.OP_SCALE, sel=dc.SEL_CHAIN, x=2, scale=1.5, path=[(3, 0)] * 9),
                              2, -1, [(2, 0)]),
    # Dense, Listing 2's a0->Lnext[q-1].Lnext[q-1].Lnext[q-1]->A
    "dense_listing2": (lambda: tg.dense_tree(8, 1000, 3, seed=4),
                       dict(kind=dc.OP_SCALE, sel=dc.SEL_CHAIN, type_=3, x=1, scale=1.25, path=[(3, 7)] * 3),
                       1, -1, [(2, 0)]),
    # the node struct, x += 0.5*y at root->child[5]->child[2]
    "node_chain_axpy": (lambda: tg.node_tree(4, 6, tg.uniform(1, 3000), seed=9),
                        dict(sel=dc.SEL_CHAIN, path=[(NODE_LEAF, 5), (NODE_LEAF, 2)]), 2, 3, [(2, 0)]),
}


@pytest.mark.parametrize("flags", [0, dc.PLAN_MAP_HOST])
@pytest.mark.parametrize("case", sorted(SELECTIVE_CASES))
def test_selective_deep_copy_of_a_chain(case, flags):
    """dc_deep_copy_selected moves only the chain's struct blocks and the op's
    arrays: the device image passes the oracle's check along the chain, an
    array off the chain still holds the bytes the buffer was filled with, the
    device walk of the chain reaches the resolved address, and the pointer
    chase and the resolved update, each followed by the copy back, give the
    oracle's host tree."""
    make, kw, xf, yf, off_chain = SELECTIVE_CASES[case]
    src, ref = make(), make()
    s = src.schema
    plan = dc.Plan(s, src.root, flags=flags)
    buf = plan.bind()
    info = plan.info
    buf[:info["data_bytes"]].fill_(0xAB)
    dop, oop = ops_pair(**kw)
    path = list(kw["path"])
    plan.deep_copy_selected(dop)
    plan.sync()
    img, base = plan.image(), plan.device_base
    ok, msg = oracle.check_chain_image(s, src.root, img, base, path, xf, yf)
    assert ok, msg
    o = plan.resolve_offset(off_chain)  # the root's first array (at least one element): not on the chain
    assert (img[o:o + 4] == 0xAB).all()
    assert not oracle.check_image(s, src.root, img, base)[0]  # not a full copy
    assert plan.verify_chain(path) == plan.resolve(path)
    for mode in ("chase", "leaf"):
        if mode == "leaf":
            plan.deep_copy_selected(dop)  # again, from the host tree the first round wrote back
        (plan.update_chase if mode == "chase" else plan.update)(dop)
        plan.copy_back()
        cp = oracle.deep_copy(s, ref.root)
        oracle.update(s, cp.root, oop)
        oracle.copy_back(s, cp.root, ref.root, oop)
        ok, msg = oracle.trees_equal(s, src.root, ref.root)
        assert ok, (mode, msg)
    plan.destroy()
    src.free()
    ref.free()



# ---- DC_PLAN_PACK_SMALL: arrays below 64 bytes at their element alignment -------------

PACKED_CASES = {
    # the pointer-heavy tree at full size: 2.2M arrays of 10 fp32 back to back
    "reloc_stress": (lambda: tg.workload("reloc_stress"), {}),
    # arrays on both sides of 64 bytes, empty ones, one-element ones
    "ragged_small": (lambda: tg.node_tree(4, 6, tg.uniform(0, 30), seed=71), {}),
    "tiny_segments": (lambda: tg.node_tree(5, 12, tg.uniform(1, 9), seed=13), {}),
    # fp64 arrays below 64 bytes: 8-byte starts
    "node64_small": (lambda: node64_tree(3, 7, tg.uniform(0, 12), seed=72), {}),
    # the Dense tree with 5 doubles per level, Listing 2's scaling on the last level
    "dense_f64_scale": (lambda: tg.dense_tree(4, 5, 3, seed=73), dict(kind=dc.OP_SCALE, type_=3, x=1, scale=1.1)),
    # one struct's small arrays by a chain: a segment that starts off a 16-byte boundary
    "chain_small": (lambda: tg.node_tree(4, 6, tg.uniform(1, 20), seed=74),
                    dict(sel=dc.SEL_CHAIN, path=[(NODE_LEAF, 5), (NODE_LEAF, 2)])),
}


@pytest.mark.parametrize("case", sorted(PACKED_CASES))
def test_packed_small_arrays(case, monkeypatch):
    """A packed plan's arena (oracle image check with the packing rule) and
    every update path on it against the oracle: the bulk-copy leaf kernel
    (with the device-side slot check), the pointer chase, the device-scan
    relocation, the persistent fused launch at each CTA size, the round trip
    (which takes its three-call path) and the direct-load leaf kernel."""
    make, kw = PACKED_CASES[case]
    P = dc.PLAN_PACK_SMALL
    full_parity(make, kw, repeat=2, flags=P, verify=True)
    full_parity(make, kw, mode="chase", flags=P)
    full_parity(make, kw, flags=P | dc.PLAN_DEVICE_SCAN)
    step_parity(make, kw, P | dc.PLAN_MAP_HOST)
    src, ref = make(), make()
    s = src.schema
    plan = dc.Plan(s, src.root, flags=P)
    plan.bind()
    dop, oop = ops_pair(**kw)
    cp = oracle.deep_copy(s, ref.root)
    plan.deep_copy()
    for threads in (128, 256, 512):  # each launch relocates again and updates once more
        plan.set_split(dop, threads, 2)
        plan.relocate_update(dop)
        plan.sync()
        oracle.update(s, cp.root, oop)
        image_ok(plan, s, cp.root)
    plan.destroy()
    src.free()
    ref.free()
    monkeypatch.setenv("DC_LEAF_TMA", "0")
    full_parity(make, kw, flags=P)


def test_packed_random_schemas_and_forest():
    rng = random.Random(7373)
    for i in range(60):
        schema, levels, rules = tg.random_schema(rng)
        full_parity(lambda: tg.Tree(schema, levels, rules, seed=700 + i), None, flags=dc.PLAN_PACK_SMALL)
    forest_parity(300, 256 << 10, "fused", flags=dc.PLAN_PACK_SMALL)


def test_packed_static_relocation_matches_dc_relocate():
    # dc_relocate_static reads the same unit-scaled tables
    t = tg.node_tree(4, 16, tg.uniform(1, 40), seed=21)
    plan = dc.Plan(t.schema, t.root, flags=dc.PLAN_PACK_SMALL)
    buf = plan.bind()
    n = plan.info["data_bytes"]
    img = np.zeros(n, dtype=np.uint8)
    for b in plan.blocks():
        if b["bytes"]:
            img[b["offset"]:b["offset"] + b["bytes"]] = np.frombuffer(ctypes.string_at(b["host"], b["bytes"]),
                                                                     dtype=np.uint8)
    image = torch.from_numpy(img).cuda()
    buf[:n].copy_(image)
    plan.relocate()
    plan.sync()
    want = buf[:n].cpu()
    ok, msg, _ = oracle.check_image(t.schema, t.root, want.numpy(), buf.data_ptr(), pack_below=PACK_BELOW)
    assert ok, msg
    buf[:n].copy_(image)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rc = dc.lib.dc_relocate_static(plan._h, buf.data_ptr(), n, status.data_ptr(),
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == 0, dc.lib.dc_last_error()
    torch.cuda.synchronize()
    assert status.item() == 0
    assert torch.equal(buf[:n].cpu(), want)
    plan.destroy()
    t.free()
