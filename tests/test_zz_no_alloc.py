"""dc_relocate_static, the relocation entry point that allocates nothing.

It serves callers that cannot allocate memory where they relocate: code whose
device memory is handed out by another application's pool (a cudaMalloc of
its own would escape that pool's accounting or fail under its cap), or a hot
path that must not allocate because cudaMalloc/cudaFree can synchronize the
whole device.  The call takes only the device data region and keeps its
scratch in a fixed array inside the library.

These tests call it through the C ABI and require the same bytes as
dc_relocate (bit for bit: relocation is integer work) on two calls in a row.
The file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import treegen as tg
import paper_1906_01128_b300 as dc

pytestmark = pytest.mark.gpu


def marshalled_image(plan) -> np.ndarray:
    """The data region as the marshal leaves it: every block copied verbatim
    (host pointers still in the slots) to its arena offset."""
    img = np.zeros(plan.info["data_bytes"], dtype=np.uint8)
    for b in plan.blocks():
        if b["bytes"]:
            img[b["offset"]:b["offset"] + b["bytes"]] = np.frombuffer(ctypes.string_at(b["host"], b["bytes"]),
                                                                     dtype=np.uint8)
    return img


def relocate_static(plan, ptr, nbytes, status):
    stream = torch.cuda.current_stream().cuda_stream
    rc = dc.lib.dc_relocate_static(plan._h, ptr, nbytes, status.data_ptr() if status is not None else None,
                                   stream)
    return rc


@pytest.mark.parametrize("make", [
    lambda: tg.workload("dense"),                       # 564 blocks, 8.7 KB of structs: two tiles
    lambda: tg.node_tree(4, 16, tg.uniform(1, 40), seed=21),  # ~13,000 blocks, 140 KB of structs: 18 tiles
], ids=["dense", "multi_tile"])
def test_static_scratch_matches_dc_relocate_twice(make):
    t = make()
    plan = dc.Plan(t.schema, t.root)
    buf = plan.bind()
    n = plan.info["data_bytes"]
    image = torch.from_numpy(marshalled_image(plan)).cuda()
    # reference: the existing entry point on the same buffer
    buf[:n].copy_(image)
    plan.relocate()
    plan.sync()
    want = buf[:n].cpu()
    ok, msg, _ = oracle.check_image(t.schema, t.root, want.numpy(), buf.data_ptr())
    assert ok, msg
    status = torch.empty(1, dtype=torch.int32, device="cuda")
    for call in range(2):
        buf[:n].copy_(image)  # back to host pointers in every slot
        status.fill_(-1)
        assert relocate_static(plan, buf.data_ptr(), n, status) == 0, dc.lib.dc_last_error()
        torch.cuda.synchronize()
        assert status.item() == 0, call
        got = buf[:n].cpu()
        assert torch.equal(got, want), f"call {call}: bytes differ from dc_relocate"
    # a buffer of the caller's own: pointers now point into that buffer
    other = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
    other[:n].copy_(image)
    assert relocate_static(plan, other.data_ptr(), n, None) == 0
    torch.cuda.synchronize()
    ok, msg, _ = oracle.check_image(t.schema, t.root, other[:n].cpu().numpy(), other.data_ptr())
    assert ok, msg
    plan.destroy()
    t.free()


def test_static_scratch_rejects_plans_beyond_its_limit():
    t = tg.node_tree(5, 16, 3, seed=1)  # 69,905 nodes: more blocks than the array holds
    plan = dc.Plan(t.schema, t.root)
    assert plan.info["nblocks"] > 65536
    dummy = torch.empty(256, dtype=torch.uint8, device="cuda")
    rc = relocate_static(plan, dummy.data_ptr(), plan.info["data_bytes"], None)
    assert dc.STATUS[rc] == "DC_EBUDGET"
    assert b"at most 65536" in dc.lib.dc_last_error()
    # 16,386 blocks, but a pointer slot in each of 16,385 tiles of 8 KiB: more tiles than the array lists
    n = 16385
    big = tg.Schema([tg.Type("Root", 16, 8, [tg.Field("n", tg.SCALAR, 0, 4),
                                              tg.Field("kids", tg.CHILD, 8, count_field=0, child_type=1)]),
                     tg.Type("Big", 8192, 8, [tg.Field("a", tg.ARRAY, 0, 4, count_const=1)])])
    kids = (ctypes.c_uint8 * (n * 8192))()
    vals = (ctypes.c_float * n)()
    ptrs = np.frombuffer(kids, dtype=np.uint64).reshape(n, 1024)
    ptrs[:, 0] = ctypes.addressof(vals) + 4 * np.arange(n, dtype=np.uint64)
    root = (ctypes.c_uint64 * 2)(n, ctypes.addressof(kids))
    p3 = dc.Plan(big, ctypes.addressof(root))
    assert p3.info["nblocks"] == n + 2
    rc = relocate_static(p3, dummy.data_ptr(), p3.info["data_bytes"], None)
    assert dc.STATUS[rc] == "DC_EBUDGET"
    assert b"relocation tiles" in dc.lib.dc_last_error()
    p3.destroy()
    small = tg.workload("tiny")
    p2 = dc.Plan(small.schema, small.root)
    rc = relocate_static(p2, dummy.data_ptr(), 256, None)  # region smaller than the plan's
    assert dc.STATUS[rc] == "DC_EINVAL"
    for x in (plan, p2):
        x.destroy()


def test_static_relocation_of_targets_64_gib_past_their_group_base():
    """Records hold a target's offset from its lane group's base in 32 bits of
    16-byte units; the plan starts a new group 2^32 units (64 GiB) past the
    base.  A 7-level Linear chain whose A arrays are 16 GiB of reserved host
    address space (never read) lays out a 120 GB arena: A_5 and A_6 lie in a
    second group.  Only the level structs (224 bytes at the start of the data
    region) are written and relocated; every slot must hold the device
    address the layout's closed form gives: level k at 32k, A_k at
    224 + k (2^34 - 16)."""
    nA, levels = 2 ** 31 - 2, 7
    t = tg.ReservedChain(levels, nA)
    plan = dc.Plan(t.schema, t.root)
    n, sb = plan.info["data_bytes"], plan.info["struct_bytes"]
    assert sb == 224 and n == 224 + levels * 8 * nA
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < n + (8 << 30):
        pytest.skip(f"needs {n / 1e9:.0f} GB of device memory, {free / 1e9:.0f} GB free")
    buf = torch.empty(n, dtype=torch.uint8, device="cuda")
    img = bytearray(sb)
    for b in plan.blocks()[:plan.info["nstruct_blocks"]]:
        img[b["offset"]:b["offset"] + b["bytes"]] = ctypes.string_at(b["host"], b["bytes"])
    buf[:sb].copy_(torch.frombuffer(img, dtype=torch.uint8))
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    assert relocate_static(plan, buf.data_ptr(), n, status) == 0, dc.lib.dc_last_error()
    torch.cuda.synchronize()
    assert status.item() == 0
    lv = np.frombuffer(buf[:sb].cpu().numpy().tobytes(), dtype=np.dtype(
        [("nA", "<i4"), ("nLnext", "<i4"), ("A", "<u8"), ("Lnext", "<u8"), ("pad", "<u8")]))
    base = buf.data_ptr()
    for k in range(levels):
        assert lv["nA"][k] == nA and lv["nLnext"][k] == (1 if k + 1 < levels else 0), k
        assert int(lv["A"][k]) == base + 224 + k * 8 * nA, k
        assert int(lv["Lnext"][k]) == (base + 32 * (k + 1) if k + 1 < levels else 0), k
    del buf
    torch.cuda.empty_cache()
    plan.destroy()
    t.free()
