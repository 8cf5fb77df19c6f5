"""Pins of the CPU oracle to facts outside itself: the paper's printed Tables 1
and 2 (through Eq 1-3), closed-form node/byte counts, hand-built trees with
hand-computed results, IEEE-754 single rounding, and planted mistakes that the
checkers must catch.  CPU only."""
import ctypes
import os
import random
from fractions import Fraction

import numpy as np
import pytest

import oracle
import treegen as tg
from treewalk import f32_view, f64_view, half_axpy_exact, i32, node_arrays, node_walk, same_bits, u64

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
UNIT = {"KB": 1024, "MB": 1024 ** 2, "GB": 1024 ** 3}


def load_table(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#") or not line.strip():
            continue
        a, b, v, u = line.split()
        rows.append((int(a), int(b), v, u))
    return rows


def fmt(nbytes, unit):
    return f"{nbytes / UNIT[unit]:.2f}"


# The paper's formulas, as printed (Eq 1, Eq 2, Eq 3).
def eq1(k, n):
    return 24 * k + 8 * n * k


def eq2(k, n):
    return 24 * k + 8 * n


def eq3(q, n, D):
    return 12 + 8 * n if D == 0 else 24 + 8 * n + q * eq3(q, n, D - 1)


def test_eq1_reproduces_table1():
    rows = load_table("paper_table1_linear_datasize.txt")
    assert len(rows) == 63
    for n, k, v, u in rows:
        assert fmt(eq1(k, n), u) == v, (n, k)


def test_eq3_reproduces_table2():
    rows = load_table("paper_table2_dense_datasize.txt")
    assert len(rows) == 40
    for n, q, v, u in rows:
        assert fmt(eq3(q, n, 3), u) == v, (n, q)


def test_oracle_count_linear_equals_table1():
    # The oracle's byte counter over generated Linear trees (24-byte level
    # struct, n doubles per level) reproduces the printed table cells.
    for n, k, v, u in load_table("paper_table1_linear_datasize.txt"):
        if n > 10 ** 5:
            continue
        t = tg.linear_tree(k, n, "allinit", seed=k)
        c = oracle.count(t.schema, t.root)
        assert c["payload_bytes"] == eq1(k, n)
        assert fmt(c["payload_bytes"], u) == v
        assert c["nstructs"] == k and c["levels"] == k
        t.free()


def test_oracle_count_linear_llinit_is_eq2():
    for k in range(2, 11):
        for n in (100, 1000, 12345):
            t = tg.linear_tree(k, n, "llinit", seed=k)
            c = oracle.count(t.schema, t.root)
            assert c["payload_bytes"] == eq2(k, n)
            # only the last level's A array exists: k structs + 1 array
            assert c["nblocks"] == k + 1
            t.free()


def test_oracle_count_dense_equals_table2():
    # Eq 3 counts the half-size last-level struct {int nA; double* A} as 12
    # bytes; its real size with padding is 16, i.e. 4 more bytes per each of
    # the q^D last-level structs.
    D = 3
    for n, q, v, u in load_table("paper_table2_dense_datasize.txt"):
        if n > 1000:
            continue
        t = tg.dense_tree(q, n, D, seed=q)
        c = oracle.count(t.schema, t.root)
        assert c["payload_bytes"] == eq3(q, n, D) + 4 * q ** D
        assert fmt(c["payload_bytes"] - 4 * q ** D, u) == v
        assert c["per_level"] == [q ** i for i in range(D + 1)]
        t.free()


@pytest.mark.parametrize("levels,fanout,n", [(4, 1, 7), (3, 16, 5), (5, 3, 11), (1, 8, 3), (6, 2, 0)])
def test_node_counts_closed_form(levels, fanout, n):
    t = tg.node_tree(levels, fanout, n, seed=3)
    c = oracle.count(t.schema, t.root)
    nodes = levels if fanout == 1 else (fanout ** levels - 1) // (fanout - 1)
    assert c["nstructs"] == nodes
    assert c["per_level"] == [fanout ** i for i in range(levels)]
    interior = nodes - fanout ** (levels - 1)
    arrays = 2 * nodes if n else 0
    assert c["nblocks"] == 1 + arrays + interior
    assert c["payload_bytes"] == 32 * nodes + nodes * 2 * 4 * n
    t.free()


def test_workload_byte_totals():
    # tiny: 4 nodes * 32 B + 4 nodes * 2 arrays * 65,536 * 4 B
    t = tg.workload("tiny")
    assert oracle.count(t.schema, t.root)["payload_bytes"] == 4 * 32 + 4 * 2 * 65536 * 4 == 2097280
    t.free()
    # deep: 64 nodes; 63 interior nodes with 2 * 1,024 floats, the leaf 2 * 2^26
    t = tg.workload("deep")
    c = oracle.count(t.schema, t.root)
    assert c["payload_bytes"] == 64 * 32 + 63 * 2 * 1024 * 4 + 2 * 2 ** 26 * 4 == 537389056
    assert c["nstructs"] == 64
    t.free()


# ---------------------------------------------------------------------------
# a hand-built node tree with known addresses
# ---------------------------------------------------------------------------

class CNode(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nchild", ctypes.c_int32), ("position", ctypes.c_void_p),
                ("velocity", ctypes.c_void_p), ("child", ctypes.c_void_p)]


def hand_tree():
    """root{n=2, nchild=2, pos=[1,2], vel=[3,4]} -> [c0{n=1, pos=[5], vel=[6]}, c1{n=0}]"""
    keep = []
    pos = (ctypes.c_float * 2)(1.0, 2.0)
    vel = (ctypes.c_float * 2)(3.0, 4.0)
    kids = (CNode * 2)()
    p0 = (ctypes.c_float * 1)(5.0)
    v0 = (ctypes.c_float * 1)(6.0)
    kids[0] = CNode(1, 0, ctypes.addressof(p0), ctypes.addressof(v0), None)
    kids[1] = CNode(0, 0, None, None, None)
    root = CNode(2, 2, ctypes.addressof(pos), ctypes.addressof(vel), ctypes.addressof(kids))
    keep += [pos, vel, kids, p0, v0, root]
    return root, keep


def test_deep_copy_hand_built_layout():
    assert ctypes.sizeof(CNode) == 32
    root, keep = hand_tree()
    s = tg.node_schema()
    cp = oracle.deep_copy(s, ctypes.addressof(root))
    b = cp.base
    # bump order: root, root.pos, root.vel, root.child[2], c0.pos, c0.vel; 16-byte starts
    assert cp.root == b
    assert (i32(b), i32(b + 4)) == (2, 2)
    assert u64(b + 8) == b + 32 and u64(b + 16) == b + 48 and u64(b + 24) == b + 64
    assert list(f32_view(b + 32, 2)) == [1.0, 2.0] and list(f32_view(b + 48, 2)) == [3.0, 4.0]
    c0, c1 = b + 64, b + 96
    assert (i32(c0), i32(c0 + 4)) == (1, 0)
    assert u64(c0 + 8) == b + 128 and u64(c0 + 16) == b + 144 and u64(c0 + 24) == 0
    assert f32_view(b + 128, 1)[0] == 5.0 and f32_view(b + 144, 1)[0] == 6.0
    assert (i32(c1), u64(c1 + 8), u64(c1 + 16), u64(c1 + 24)) == (0, 0, 0, 0)
    assert cp.used == 148
    # nothing in the copy points back into the source
    src_ptrs = {root.position, root.velocity, root.child}
    assert not src_ptrs & {u64(b + 8), u64(b + 16), u64(b + 24)}


def test_deep_copy_relative_pointer_base():
    root, keep = hand_tree()
    s = tg.node_schema()
    base = 0x7A0000000000
    cp = oracle.deep_copy(s, ctypes.addressof(root), ptr_base=base)
    b = cp.base
    assert u64(b + 8) == base + 32 and u64(b + 24) == base + 64 and u64(b + 64 + 8) == base + 128


def test_resolve_hand_built():
    root, keep = hand_tree()
    s = tg.node_schema()
    r = ctypes.addressof(root)
    assert oracle.host_resolve(s, r, []) == r
    assert oracle.host_resolve(s, r, [(4, 1)]) == root.child + 32
    assert oracle.host_resolve(s, r, [(4, 0), (2, 0)]) == ctypes.cast(root.child, ctypes.POINTER(CNode))[0].position
    assert oracle.host_resolve(s, r, [(3, 1)]) == root.velocity + 4
    with pytest.raises(RuntimeError):
        oracle.host_resolve(s, r, [(4, 2)])
    with pytest.raises(RuntimeError):
        oracle.host_resolve(s, r, [(4, 1), (2, 0)])  # c1 has no elements
    base = 0x7A0000000000
    cp = oracle.deep_copy(s, r, ptr_base=base)
    img = cp.image()
    assert oracle.image_resolve(s, img, base, []) == base
    assert oracle.image_resolve(s, img, base, [(4, 1)]) == base + 96
    assert oracle.image_resolve(s, img, base, [(4, 0), (2, 0)]) == base + 128
    assert oracle.image_resolve(s, img, base, [(4, 0), (3, 0)]) == base + 144
    assert oracle.image_resolve(s, img, base, [(2, 1)]) == base + 36


def test_resolve_listing1_chain():
    # simulation->atoms->traits->positions (Listing 1)
    t = tg.listing1_tree(10, seed=4)
    s = t.schema
    atoms = u64(t.root + 8)
    traits = u64(atoms + 8)
    pos0 = u64(traits + 8)
    assert oracle.host_resolve(s, t.root, [(1, 0), (1, 0), (1, 0)]) == pos0
    base = 0x7B0000000000
    cp = oracle.deep_copy(s, t.root, ptr_base=base)
    got = oracle.image_resolve(s, cp.image(), base, [(1, 0), (1, 0), (1, 0)])
    off = got - base
    assert cp.image()[off:off + 80].tobytes() == ctypes.string_at(pos0, 80)
    t.free()


# ---------------------------------------------------------------------------
# the leaf update: single IEEE-754 rounding, hand-computed special cases
# ---------------------------------------------------------------------------

def test_update_special_values():
    keep = []
    vals_p = [1.0, 0.25, -0.5, 2.0 ** -23, 1.0, 1.0 + 2.0 ** -23, -1.0, 0.75]
    vals_v = [-2.0, 0.5, 1.0, 2.0 ** -23, 2.0 ** -23, 2.0 ** -23, -2.0 ** -23, 0.0]
    # hand-computed: 1-1=0; 0.25+0.25; -0.5+0.5=0; 2^-23+2^-24; 1+2^-24 ties to
    # even -> 1; (1+2^-23)+2^-24 ties to even -> 1+2^-22; -1-2^-24 -> -1 (even);
    # 0.75+0
    want = [0.0, 0.5, 0.0, 1.5 * 2.0 ** -23, 1.0, 1.0 + 2.0 ** -22, -1.0, 0.75]
    n = len(vals_p)
    pos = (ctypes.c_float * n)(*vals_p)
    vel = (ctypes.c_float * n)(*vals_v)
    root = CNode(n, 0, ctypes.addressof(pos), ctypes.addressof(vel), None)
    keep += [pos, vel]
    s = tg.node_schema()
    oracle.update(s, ctypes.addressof(root), oracle.Op())
    got = np.frombuffer(bytes(pos), dtype=np.float32)
    assert list(got) == [np.float32(w) for w in want]
    assert np.signbit(got[0]) == False and np.signbit(got[2]) == False  # RN: x + (-x) = +0
    assert list(np.frombuffer(bytes(vel), dtype=np.float32)) == [np.float32(v) for v in vals_v]


@pytest.mark.parametrize("levels,fanout,n", [(4, 1, 1000), (3, 5, 77), (2, 16, 257)])
def test_update_all_is_single_rounding(levels, fanout, n):
    t = tg.node_tree(levels, fanout, n, seed=levels * 31 + fanout)
    s = t.schema
    before = node_arrays(t.root)
    cp = oracle.deep_copy(s, t.root)
    oracle.update(s, cp.root, oracle.Op())
    after = node_arrays(cp.root)
    assert before.keys() == after.keys()
    for path, (p, v) in before.items():
        p2, v2 = after[path]
        assert same_bits(p2, half_axpy_exact(p, v)), path
        assert same_bits(v2, v)
    t.free()


def test_update_chain_touches_one_node():
    t = tg.node_tree(3, 4, 33, seed=9)
    s = t.schema
    before = node_arrays(t.root)
    cp = oracle.deep_copy(s, t.root)
    path = [(4, 3), (4, 1)]
    oracle.update(s, cp.root, oracle.Op(sel=oracle.SEL_CHAIN, path=path))
    after = node_arrays(cp.root)
    for p, (x, y) in before.items():
        want = half_axpy_exact(x, y) if p == (3, 1) else x
        assert same_bits(after[p][0], want), p
    t.free()


def test_scale_f64_is_correctly_rounded():
    # The paper's scaling kernel (Sec. 4.1.2; Listing 2) on the Linear shape.
    t = tg.linear_tree(3, 200, "allinit", seed=5)
    s = t.schema
    srcA = []
    a = t.root
    while a:
        srcA.append(f64_view(u64(a + 8), 200).copy())
        a = u64(a + 16)
    cp = oracle.deep_copy(s, t.root)
    oracle.update(s, cp.root, oracle.Op(kind=oracle.OP_SCALE, x_field=2, scale=1.5))
    a = cp.root
    for want_src in srcA:
        got = f64_view(u64(a + 8), 200)
        exact = [float(Fraction(float(x)) * Fraction(3, 2)) for x in want_src]
        assert list(got) == exact
        a = u64(a + 16)
    t.free()


def test_scale_listing2_chain_last_element():
    # a0->Lnext[q-1].Lnext[q-1].Lnext[q-1].A[i] *= scale: only that A changes
    q, n, D = 3, 17, 3
    t = tg.dense_tree(q, n, D, seed=2)
    s = t.schema
    path = [(3, q - 1)] * D
    target_src = oracle.host_resolve(s, t.root, path + [(1, 0)])
    want = [float(Fraction(float(x)) * Fraction(5, 4)) for x in f64_view(target_src, n)]
    cp = oracle.deep_copy(s, t.root)
    op = oracle.Op(kind=oracle.OP_SCALE, sel=oracle.SEL_CHAIN, path=path, type=D, x_field=1, scale=1.25)
    oracle.update(s, cp.root, op)
    target = oracle.host_resolve(s, cp.root, path + [(1, 0)])
    assert list(f64_view(target, n)) == want
    # every other A is untouched: copy back only that array, then compare trees
    t2 = tg.dense_tree(q, n, D, seed=2)
    oracle.copy_back(s, cp.root, t2.root, op)
    ok, msg = oracle.trees_equal(s, t2.root, cp.root)
    assert ok, msg
    ok, msg = oracle.trees_equal(s, t.root, t2.root)
    assert not ok
    t.free()
    t2.free()


def f32_round(fr: Fraction) -> np.float32:
    """The fp32 value nearest to the exact rational `fr` (ties to even), for
    rationals that a double holds exactly (products of two fp32 values): the
    double conversion is then exact and the fp32 cast is the one rounding."""
    d = float(fr)
    assert Fraction(d) == fr, "not exact in a double"
    return np.float32(d)


@pytest.mark.parametrize("scale", [1.1, -0.7, 1.0 / 3.0])
def test_scale_f32_uses_the_scale_rounded_to_float(scale):
    # The paper's scaling kernel (Sec. 4.1.2, Listing 2) on fp32 arrays: the
    # scale is an fp32 operand, so x*scale is the exact product of x and
    # float(scale), rounded once to fp32.  Scales that are not fp32 numbers
    # separate this from multiplying by the double and rounding twice.
    t = tg.node_tree(3, 4, 777, seed=21)
    s = t.schema
    before = node_arrays(t.root)
    cp = oracle.deep_copy(s, t.root)
    oracle.update(s, cp.root, oracle.Op(kind=oracle.OP_SCALE, x_field=2, scale=scale))
    after = node_arrays(cp.root)
    sf = Fraction(float(np.float32(scale)))
    differs = 0
    for path, (p, v) in before.items():
        want = np.array([f32_round(Fraction(float(x)) * sf) for x in p], dtype=np.float32)
        assert same_bits(after[path][0], want), path
        assert same_bits(after[path][1], v), path  # velocity is not an operand
        twice = (p.astype(np.float64) * scale).astype(np.float32)  # the double product, rounded again
        differs += int((twice != want).sum())
    assert differs > 100  # the pin tells the two readings apart
    t.free()


class CTraits(ctypes.Structure):
    """Listing 1's Traits struct: {int n; double* positions0..2}, 32 bytes."""
    _fields_ = [("n", ctypes.c_int32), ("pad", ctypes.c_int32), ("p0", ctypes.c_void_p), ("p1", ctypes.c_void_p),
                ("p2", ctypes.c_void_p)]


def test_axpy_f64_special_values():
    # x + 0.5*y in fp64 with each operation rounded once (ties to even), values
    # computed by hand.  Halving is exact except below the normal range, where
    # the product itself rounds: 0.5 * 2^-1074 is a tie between 0 and 2^-1074,
    # and goes to 0.
    e = 2.0 ** -52
    tiny = 2.0 ** -1074
    xs = [1.0, 1.0 + e, -1.0, 0.25, 0.75, tiny, 3.0, -0.5]
    ys = [e, e, -e, -0.5, 0.5, tiny, 2.0 ** 53, 1.0]
    # 1 + 2^-53: tie -> 1 (even); 1 + 2^-52 + 2^-53: tie -> 1 + 2^-51 (even);
    # -1 - 2^-53 -> -1; 0.25 - 0.25 = +0; 0.75 + 0.25 = 1; 2^-1074 + 0;
    # 3 + 2^52 is exact; -0.5 + 0.5 = +0
    want = [1.0, 1.0 + 2 * e, -1.0, 0.0, 1.0, tiny, 3.0 + 2.0 ** 52, 0.0]
    n = len(xs)
    x = (ctypes.c_double * n)(*xs)
    y = (ctypes.c_double * n)(*ys)
    z = (ctypes.c_double * n)(*([7.0] * n))
    node = CTraits(n, 0, ctypes.addressof(x), ctypes.addressof(y), ctypes.addressof(z))
    s = tg.Schema([tg.listing1_schema().types[2]])
    oracle.update(s, ctypes.addressof(node), oracle.Op(kind=oracle.OP_AXPY_HALF, type=0, x_field=1, y_field=2))
    got = np.frombuffer(bytes(x), dtype=np.float64)
    assert [float(g) for g in got] == want
    assert not np.signbit(got[3]) and not np.signbit(got[7])  # RN: a + (-a) = +0
    assert list(np.frombuffer(bytes(y), dtype=np.float64)) == ys
    assert list(np.frombuffer(bytes(z), dtype=np.float64)) == [7.0] * n


@pytest.mark.parametrize("sel", ["all", "chain"])
def test_axpy_f64_is_correctly_rounded(sel):
    # Listing 1's Simulation->Atoms->Traits chain with positions0 += 0.5 *
    # positions1 in fp64: the generated values are multiples of 2^-52 in
    # [-1, 1), so halving is exact and each result is the exact sum rounded once
    # (Python's int/int division, under float(Fraction), rounds correctly).
    t = tg.listing1_tree(3000, seed=23)
    s = t.schema
    traits = oracle.host_resolve(s, t.root, [(1, 0), (1, 0)])
    x0, y0, z0 = (f64_view(u64(traits + off), 3000).copy() for off in (8, 16, 24))
    cp = oracle.deep_copy(s, t.root)
    op = oracle.Op(kind=oracle.OP_AXPY_HALF, type=2, x_field=1, y_field=2)
    if sel == "chain":
        op = oracle.Op(kind=oracle.OP_AXPY_HALF, sel=oracle.SEL_CHAIN, path=[(1, 0), (1, 0)], type=2, x_field=1,
                       y_field=2)
    oracle.update(s, cp.root, op)
    ct = oracle.host_resolve(s, cp.root, [(1, 0), (1, 0)])
    x1, y1, z1 = (f64_view(u64(ct + off), 3000) for off in (8, 16, 24))
    want = np.array([float(Fraction(float(a)) + Fraction(float(b)) / 2) for a, b in zip(x0, y0)])
    assert same_bits(x1, want)
    assert same_bits(y1, y0) and same_bits(z1, z0)
    rounded = sum(Fraction(float(a)) + Fraction(float(b)) / 2 != Fraction(float(w)) for a, b, w in zip(x0, y0, want))
    # sums at or above 1 in magnitude whose exact value needs 54 bits round:
    # about one in fourteen here, enough to exercise ties and rounding
    assert rounded > 100
    t.free()


# ---------------------------------------------------------------------------
# copy back and the results check
# ---------------------------------------------------------------------------

def test_copy_back_writes_only_positions():
    t = tg.node_tree(3, 3, 50, seed=12)
    ref = tg.node_tree(3, 3, 50, seed=12)  # same seed: an untouched twin
    s = t.schema
    cp = oracle.deep_copy(s, t.root)
    oracle.update(s, cp.root, oracle.Op())
    oracle.copy_back(s, cp.root, t.root, oracle.Op())
    a, r = node_arrays(t.root), node_arrays(ref.root)
    for path in r:
        assert same_bits(a[path][0], half_axpy_exact(*r[path]))
        assert same_bits(a[path][1], r[path][1])
    # scalars and padding untouched, host pointers untouched
    for na, nr in zip(node_walk(t.root), node_walk(ref.root)):
        assert na["raw"][:8] == nr["raw"][:8]
    t.free()
    ref.free()


def test_trees_equal_detects_planted_differences():
    s = tg.node_schema()
    a = tg.node_tree(3, 3, 20, seed=7)
    b = tg.node_tree(3, 3, 20, seed=7)
    assert oracle.trees_equal(s, a.root, b.root)[0]
    nodes = list(node_walk(b.root))
    # one float in a leaf array
    f32_view(nodes[5]["pos"], 20)[13] += np.float32(2.0 ** -20)
    ok, msg = oracle.trees_equal(s, a.root, b.root)
    assert not ok and "array differs" in msg
    f32_view(nodes[5]["pos"], 20)[13] -= np.float32(2.0 ** -20)
    assert oracle.trees_equal(s, a.root, b.root)[0]
    # a scalar: a child count one higher than the twin's
    cnt = ctypes.c_int32.from_address(nodes[2]["addr"])
    cnt.value -= 1
    ok, msg = oracle.trees_equal(s, a.root, b.root)
    assert not ok and "struct byte" in msg
    cnt.value += 1
    c = tg.node_tree(3, 3, 20, seed=8)
    assert not oracle.trees_equal(s, a.root, c.root)[0]
    for t in (a, b, c):
        t.free()


def _image_setup():
    t = tg.node_tree(3, 3, 9, seed=21)
    base = 0x7C0000000000
    cp = oracle.deep_copy(t.schema, t.root, ptr_base=base)
    return t, base, cp


def test_check_image_accepts_a_correct_copy():
    t, base, cp = _image_setup()
    ok, msg, seen = oracle.check_image(t.schema, t.root, cp.image(), base)
    assert ok, msg
    c = oracle.count(t.schema, t.root)
    for k in ("nstructs", "nblocks", "payload_bytes", "nptr"):
        assert seen[k] == c[k]
    t.free()


def _plant(img, off, value):
    img[off:off + 8] = np.frombuffer(int(value).to_bytes(8, "little"), dtype=np.uint8)


@pytest.mark.parametrize("mistake", ["leaf_byte", "ptr_plus16", "ptr_to_source", "shared_block",
                                     "outside", "misaligned", "scalar", "null_with_count",
                                     "nonnull_count0"])
def test_check_image_catches_planted_mistakes(mistake):
    t, base, cp = _image_setup()
    img = cp.image().copy()
    s = t.schema
    rel = lambda p: p - base  # noqa: E731
    rp = int.from_bytes(img[8:16].tobytes(), "little")      # root.position
    rv = int.from_bytes(img[16:24].tobytes(), "little")     # root.velocity
    rc = int.from_bytes(img[24:32].tobytes(), "little")     # root.child
    if mistake == "leaf_byte":
        img[rel(rv) + 5] ^= 1
    elif mistake == "ptr_plus16":
        _plant(img, 8, rp + 16)
    elif mistake == "ptr_to_source":
        _plant(img, 8, u64(t.root + 8))
    elif mistake == "shared_block":
        _plant(img, 16, rp)  # velocity now points at position's block
    elif mistake == "outside":
        _plant(img, 8, base + len(img) + 64)
    elif mistake == "misaligned":
        _plant(img, rel(rc) + 8, int.from_bytes(img[rel(rc) + 8:rel(rc) + 16].tobytes(), "little") + 4)
    elif mistake == "scalar":
        img[rel(rc) + 32 + 4] ^= 1  # child[1].nchild
    elif mistake == "null_with_count":
        _plant(img, rel(rc) + 16, 0)
    elif mistake == "nonnull_count0":
        # a leaf's child pointer must stay NULL (its count is 0)
        leaf = rel(int.from_bytes(img[rel(rc) + 24:rel(rc) + 32].tobytes(), "little"))
        _plant(img, leaf + 24, base)
    ok, msg, _ = oracle.check_image(s, t.root, img, base)
    assert not ok, mistake
    t.free()


# ---------------------------------------------------------------------------
# the image of a selective deep copy of one chain (Sec. 2)
# ---------------------------------------------------------------------------

def _le(img, off, n=8, signed=False):
    return int.from_bytes(img[off:off + n].tobytes(), "little", signed=signed)


def _dense_chain():
    """The Dense tree (Fig 4) with q = 4, D = 3 and Listing 2's chain
    a0->Lnext[q-1].Lnext[q-1].Lnext[q-1]; returns the tree, a full deep copy's
    image at a device-like base, the path and the byte spans a selective copy
    of that chain holds (the root struct, each Lnext block on the path, the
    last struct's A array), found by reading the image by hand."""
    q, D = 4, 3
    t = tg.dense_tree(q, 50, D, seed=31)
    base = 0x7D0000000000
    img = oracle.deep_copy(t.schema, t.root, ptr_base=base).image().copy()
    path = [(3, q - 1)] * D
    spans, off = [(0, 24)], 0
    for k in range(D):
        b = _le(img, off + 16) - base  # Lnext of an L0..L(D-1) struct (offset 16)
        size = 24 if k + 1 < D else 16  # the last level is the half-size struct
        spans.append((b, b + q * size))
        off = b + (q - 1) * size
    a, n = _le(img, off + 8) - base, _le(img, off, 4, signed=True)  # {int nA; double* A}
    spans.append((a, a + 8 * n))
    return t, base, img, path, spans, D


def test_chain_image_accepts_a_selective_copy_and_nothing_else_is_read():
    t, base, img, path, spans, D = _dense_chain()
    s = t.schema
    ok, msg = oracle.check_chain_image(s, t.root, img, base, path, x_field=1)
    assert ok, msg
    # overwrite every byte off the chain: the chain check still passes, the
    # full deep-copy check does not
    sel = np.full_like(img, 0xAB)
    for lo, hi in spans:
        sel[lo:hi] = img[lo:hi]
    assert sum(hi - lo for lo, hi in spans) < len(img) // 10
    ok, msg = oracle.check_chain_image(s, t.root, sel, base, path, x_field=1)
    assert ok, msg
    assert not oracle.check_image(s, t.root, sel, base)[0]
    # a mistake off the chain is not looked at: the root's own A array
    sel[_le(img, 8) - base + 3] ^= 1
    assert oracle.check_chain_image(s, t.root, sel, base, path, x_field=1)[0]
    t.free()


@pytest.mark.parametrize("mistake", ["array_byte", "path_struct_byte", "sibling_struct_byte", "ptr_plus16",
                                     "ptr_to_source", "outside", "misaligned_array", "short_block"])
def test_chain_image_catches_planted_mistakes(mistake):
    t, base, img, path, spans, D = _dense_chain()
    s = t.schema
    (r0, _), (b1, _), (b2, _), (b3, _), (a, a_end) = spans
    if mistake == "array_byte":
        img[a + 13] ^= 1
    elif mistake == "path_struct_byte":
        img[b2 + 3 * 24 + 4] ^= 1  # Lnext[3].Lnext[3].nLnext
    elif mistake == "sibling_struct_byte":
        img[b1 + 0] ^= 1  # Lnext[0].nA: off the path, in a block the chain passes through
    elif mistake == "ptr_plus16":
        _plant(img, b1 + 3 * 24 + 16, _le(img, b1 + 3 * 24 + 16) + 16)
    elif mistake == "ptr_to_source":
        _plant(img, 16, u64(t.root + 16))  # the root's Lnext still the host's
    elif mistake == "outside":
        _plant(img, b3 + 3 * 16 + 8, base + len(img) - 8)  # the last struct's A runs past the arena
    elif mistake == "misaligned_array":
        _plant(img, b3 + 3 * 16 + 8, base + a + 8)
    elif mistake == "short_block":
        _plant(img, 16, base + len(img) - 2 * 24)  # room for 2 of the root's 4 children
    ok, msg = oracle.check_chain_image(s, t.root, img, base, path, x_field=1)
    assert not ok, mistake
    t.free()


def test_chain_image_with_x_and_y_on_a_node_chain():
    # the node struct's chain root->child[2]->child[1] with x = position, y = velocity
    t = tg.node_tree(3, 3, 40, seed=22)
    s = t.schema
    base = 0x7E0000000000
    img = oracle.deep_copy(s, t.root, ptr_base=base).image().copy()
    path = [(4, 2), (4, 1)]
    assert oracle.check_chain_image(s, t.root, img, base, path, x_field=2, y_field=3)[0]
    vel = oracle.image_resolve(s, img, base, path + [(3, 0)]) - base
    img[vel + 7] ^= 1  # the chain's y array
    assert not oracle.check_chain_image(s, t.root, img, base, path, x_field=2, y_field=3)[0]
    assert oracle.check_chain_image(s, t.root, img, base, path, x_field=2)[0]  # y not asked for
    t.free()


@pytest.mark.parametrize("case", ["f32_small_4", "f32_small_2", "f64_small_4", "f64_small_8", "f32_large_4"])
def test_check_image_packed_alignment(case):
    # The packed layout's promise: an array of fewer than 64 bytes may start on
    # its element alignment (8 bytes for f64, else 4); every other block on 16.
    # Move the root's first array up into its padding and check both readings.
    if case.startswith("f32"):
        n = 10 if "small" in case else 17           # 40 B (8 B of padding) or 68 B (12 B of padding)
        t = tg.node_tree(2, 3, n, seed=41)
        field_off, nbytes = 8, 4 * n               # Node.position
    else:
        t = tg.linear_tree(2, 5, "allinit", seed=42)  # A: 5 doubles = 40 B
        field_off, nbytes = 8, 40
    by = int(case.rsplit("_", 1)[1])
    base = 0x7F0000000000
    img = oracle.deep_copy(t.schema, t.root, ptr_base=base).image().copy()
    p = int.from_bytes(img[field_off:field_off + 8].tobytes(), "little")
    o = p - base
    assert o % 16 == 0
    img[o + by:o + by + nbytes] = img[o:o + nbytes].copy()
    _plant(img, field_off, p + by)
    s = t.schema
    assert not oracle.check_image(s, t.root, img, base)[0]  # 16-byte blocks everywhere
    ok = oracle.check_image(s, t.root, img, base, pack_below=64)[0]
    assert ok == (case in ("f32_small_4", "f64_small_8")), case
    t.free()


def test_random_schemas_copy_and_image_agree():
    rng = random.Random(1234)
    for i in range(150):
        schema, levels, rules = tg.random_schema(rng)
        t = tg.Tree(schema, levels, rules, seed=i)
        c = oracle.count(schema, t.root)
        assert c["payload_bytes"] == t.payload_bytes and c["nblocks"] == t.nblocks
        cp = oracle.deep_copy(schema, t.root)
        ok, msg = oracle.trees_equal(schema, t.root, cp.root)
        assert ok, msg
        base = 0x7D0000000000
        img = oracle.deep_copy(schema, t.root, ptr_base=base)
        ok, msg, seen = oracle.check_image(schema, t.root, img.image(), base)
        assert ok, msg
        assert seen["nblocks"] == c["nblocks"]
        t.free()


def test_generator_is_deterministic():
    s = tg.node_schema()
    a = tg.workload("tiny")
    b = tg.workload("tiny")
    c = tg.workload("tiny", seed=99)
    assert oracle.trees_equal(s, a.root, b.root)[0]
    assert not oracle.trees_equal(s, a.root, c.root)[0]
    # values are multiples of 2^-23 in [-1, 1)
    v = node_arrays(a.root)[()][0]
    assert v.min() >= -1.0 and v.max() < 1.0
    assert np.all(np.ldexp(v.astype(np.float64), 23) == np.round(np.ldexp(v.astype(np.float64), 23)))
    for t in (a, b, c):
        t.free()


PARALLEL_CASES = [
    # (tree, op): f32 axpy over every node with multi-chunk and empty arrays; f64 scale over every
    # level and on a chain; an axpy on one node reached by a chain
    (lambda: tg.node_tree(3, 5, tg.uniform(0, 200000), seed=31), oracle.Op()),
    (lambda: tg.linear_tree(5, 150001, "allinit", seed=32), oracle.Op(kind=oracle.OP_SCALE, x_field=2, scale=1.5)),
    (lambda: tg.linear_tree(6, 70000, "llinit", seed=33),
     oracle.Op(kind=oracle.OP_SCALE, sel=oracle.SEL_CHAIN, x_field=2, scale=-0.75, path=[(3, 0)] * 5)),
    (lambda: tg.node_tree(3, 4, tg.uniform(1, 90000), seed=34),
     oracle.Op(sel=oracle.SEL_CHAIN, path=[(4, 3), (4, 1)])),
]


@pytest.mark.parametrize("threads", [1, 3, 0])
@pytest.mark.parametrize("case", range(len(PARALLEL_CASES)))
def test_parallel_update_equals_the_sequential_update(case, threads):
    """The multi-core CPU baseline (update_parallel) is pinned to the oracle's
    update: on the same inputs every array is bit-identical afterwards, for
    any thread count."""
    make, op = PARALLEL_CASES[case]
    a, b = make(), make()
    oracle.update(a.schema, a.root, op)
    oracle.update_parallel(b.schema, b.root, op, threads)
    ok, msg = oracle.trees_equal(a.schema, a.root, b.root)
    assert ok, msg
    a.free()
    b.free()
