"""Debug switches read from the environment, exercised without faulting a GPU.

- DC_FAULT_HOST_ALLOC=1: every pinned host allocation fails as if page-locked
  memory had run out.  Binding a plan, creating a host arena and creating a
  server report DC_ENOMEM; once the switch is off, the same plan binds and its
  deep copy, update and copy back match the oracle.
- DC_DEBUG=1: plans run with DC_PLAN_VERIFY.  The first relocation after a
  deep copy passes the device-side check; relocating the same arena again
  finds device addresses where the check expects the host's, and dc_sync
  reports DC_EVERIFY.
- DC_WAIT_LIMIT=0: the first mbarrier wait of every pipeline step of the
  bulk-copy kernels gives up at once.  Each kernel records DC_ETIMEOUT, waits
  (at the full limit) for the bulk copies it has in flight, and returns; the
  status reaches the host through dc_sync and the context stays usable: with
  the switch off, the same plan's deep copy, update and copy back match the
  oracle.
"""
import pytest
import torch

import oracle
import treegen as tg
import paper_1906_01128_b300 as dc

pytestmark = pytest.mark.gpu


def full_check(s, t, p):
    ref = tg.workload("tiny")
    p.deep_copy()
    p.sync()
    ok, msg, _ = oracle.check_image(s, t.root, p.image(), p.device_base)
    assert ok, msg
    p.update(dc.Op())
    p.copy_back()
    cp = oracle.deep_copy(s, ref.root)
    oracle.update(s, cp.root, oracle.Op())
    oracle.copy_back(s, cp.root, ref.root, oracle.Op())
    ok, msg = oracle.trees_equal(s, t.root, ref.root)
    assert ok, msg


def test_pinned_allocation_failures_are_reported(monkeypatch):
    t = tg.workload("tiny")
    s = t.schema
    p = dc.Plan(s, t.root)
    monkeypatch.setenv("DC_FAULT_HOST_ALLOC", "1")
    with pytest.raises(dc.DcError) as e:
        p.bind()
    assert e.value.name == "DC_ENOMEM"
    with pytest.raises(dc.DcError) as e:
        dc.HostArena(1 << 20)
    assert e.value.name == "DC_ENOMEM"
    pool = torch.empty(8 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(dc.DcError) as e:
        dc.Server(s, pool, pinned_bytes=8 << 20, slots=2)
    assert e.value.name == "DC_ENOMEM"
    monkeypatch.delenv("DC_FAULT_HOST_ALLOC")
    p.bind()  # the same plan, once pinned memory is there
    full_check(s, t, p)
    p.destroy()


def test_debug_switch_turns_on_verification(monkeypatch):
    monkeypatch.setenv("DC_DEBUG", "1")
    t = tg.workload("tiny")
    s = t.schema
    p = dc.Plan(s, t.root)
    p.bind()
    full_check(s, t, p)  # the first relocation after a deep copy passes the check
    p.relocate()  # the slots now hold device addresses, not the recorded host ones
    with pytest.raises(dc.DcError) as e:
        p.sync()
    assert e.value.name == "DC_EVERIFY"
    p.destroy()


def _timeout_then_parity(kernel, monkeypatch):
    make = lambda: tg.node_tree(3, 16, tg.uniform(1, 5000), seed=51)  # 273 nodes, 4 relocation tiles' worth of slots
    src, ref = make(), make()
    s = src.schema
    p = dc.Plan(s, src.root)
    p.bind()
    op = dc.Op()
    if kernel != "relocate":
        p.deep_copy()
        p.sync()
    monkeypatch.setenv("DC_WAIT_LIMIT", "0")
    {"relocate": p.deep_copy, "leaf_tma": lambda: p.update(op), "fused": lambda: p.relocate_update(op)}[kernel]()
    with pytest.raises(dc.DcError) as e:
        p.sync()
    assert e.value.name == "DC_ETIMEOUT"
    p.sync()  # the status was reported once and cleared
    monkeypatch.delenv("DC_WAIT_LIMIT")
    p.deep_copy()  # start again from the host tree, at the default limit
    p.sync()
    ok, msg, _ = oracle.check_image(s, src.root, p.image(), p.device_base)
    assert ok, msg
    if kernel == "fused":
        p.relocate_update(op)
    else:
        p.update(op)
    p.copy_back()
    cp = oracle.deep_copy(s, ref.root)
    oracle.update(s, cp.root, oracle.Op())
    oracle.copy_back(s, cp.root, ref.root, oracle.Op())
    ok, msg = oracle.trees_equal(s, src.root, ref.root)
    assert ok, msg
    p.destroy()


@pytest.mark.parametrize("kernel", ["relocate", "leaf_tma", "fused"])
def test_a_wait_that_runs_out_reports_a_timeout(kernel, monkeypatch):
    monkeypatch.delenv("DC_LEAF_TMA", raising=False)  # the bulk-copy leaf kernel
    _timeout_then_parity(kernel, monkeypatch)
