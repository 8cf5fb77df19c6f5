"""Seeded synthetic inputs for the deep-copy benchmarks (shared by the CPU
oracle and the CUDA path; holds none of the deep-copy arithmetic).

A *schema* describes C struct types by field offsets: SCALAR (a signed 4- or
8-byte integer), ARRAY (a pointer to `count` primitive elements) and CHILD (a
pointer to a contiguous array of `count` structs).  `build()` materialises one
host tree of malloc'd blocks with the C generator in ``treegen.c``.

Named workloads (node struct ``{int32 n; int32 nchild; float* position;
float* velocity; Node* child}``, 32 bytes):

=============  =====================================================================
tiny           linear chain, 4 levels, n = 65,536 per node            (seed 1)
dense          3 levels, fanout 16 (273 nodes), n ~ lognormal(65,536, sigma 1.2),
               capped at 4,194,304                                      (seed 2)
deep           linear chain, 64 levels, n = 1,024 inside, 2^26 at the leaf (seed 3)
reloc_stress   6 levels, fanout 16 (1,118,481 nodes), n = 10            (seed 6)
=============  =====================================================================

The paper's own shapes are also provided: the Linear scenario (Fig 3, struct
``{int nA; int nLnext; double* A; L* Lnext}``), the Dense scenario (Fig 4, with
a 16-byte last-level struct ``{int nA; double* A}``) and the three-type chain of
Listing 1 (``simulation->atoms->traits->positions``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field as dc_field
from typing import List, Optional, Sequence

SCALAR, ARRAY, CHILD = 0, 1, 2
F32, F64, BYTES = 0, 1, 2
CONST, UNIFORM, LOGNORMAL = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libtreegen.so")


def build_lib(force: bool = False) -> str:
    """Compile ``libtreegen.so`` in place (gcc, no CUDA)."""
    src = os.path.join(_HERE, "treegen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "treegen.h"))):
        subprocess.check_call(["gcc", "-O2", "-Wall", "-fPIC", "-shared", "-pthread",
                               "-o", _SO, src, "-lm"])
    return _SO


class _Field(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("offset", ctypes.c_uint32),
                ("elem_size", ctypes.c_uint32), ("count_field", ctypes.c_int32),
                ("count_const", ctypes.c_uint64), ("child_type", ctypes.c_int32),
                ("elem_kind", ctypes.c_int32)]


class _Type(ctypes.Structure):
    _fields_ = [("size", ctypes.c_uint32), ("align", ctypes.c_uint32),
                ("nfields", ctypes.c_uint32), ("fields", ctypes.POINTER(_Field))]


class _Schema(ctypes.Structure):
    _fields_ = [("ntypes", ctypes.c_uint32), ("root_type", ctypes.c_uint32),
                ("types", ctypes.POINTER(_Type))]


class _Dist(ctypes.Structure):
    _fields_ = [("dist", ctypes.c_int32), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("c", ctypes.c_double)]


class _Rule(ctypes.Structure):
    _fields_ = [("type", ctypes.c_uint32), ("field", ctypes.c_uint32),
                ("interior", _Dist), ("leaf", _Dist)]


class _Shape(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_uint32), ("nrules", ctypes.c_uint32),
                ("rules", ctypes.POINTER(_Rule)), ("nthreads", ctypes.c_uint32)]


_lib_handle = None


def lib():
    global _lib_handle
    if _lib_handle is None:
        L = ctypes.CDLL(build_lib())
        L.tg_build.restype = ctypes.c_void_p
        L.tg_build.argtypes = [ctypes.POINTER(_Schema), ctypes.POINTER(_Shape), ctypes.c_uint64]
        L.tg_build_ex.restype = ctypes.c_void_p
        L.tg_build_ex.argtypes = [ctypes.POINTER(_Schema), ctypes.POINTER(_Shape), ctypes.c_uint64,
                                  ctypes.c_void_p, ctypes.c_void_p]
        L.tg_dry_bytes.restype = ctypes.c_int
        L.tg_dry_bytes.argtypes = [ctypes.POINTER(_Schema), ctypes.POINTER(_Shape), ctypes.c_uint64,
                                   ctypes.POINTER(ctypes.c_uint64)]
        for name in ("tg_payload_bytes", "tg_nstructs", "tg_nblocks"):
            getattr(L, name).restype = ctypes.c_uint64
            getattr(L, name).argtypes = [ctypes.c_void_p]
        L.tg_nelems.restype = ctypes.c_uint64
        L.tg_nelems.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32]
        L.tg_root.restype = ctypes.c_void_p
        L.tg_root.argtypes = [ctypes.c_void_p]
        L.tg_free.restype = None
        L.tg_free.argtypes = [ctypes.c_void_p]
        L.tg_error.restype = ctypes.c_char_p
        _lib_handle = L
    return _lib_handle


# ---------------------------------------------------------------------------
# schema description (plain data; each C library mirrors it in its own struct)
# ---------------------------------------------------------------------------

@dataclass
class Field:
    name: str
    kind: int
    offset: int
    elem_size: int = 0
    count_field: int = -1
    count_const: int = 0
    child_type: int = -1
    elem_kind: int = F32


@dataclass
class Type:
    name: str
    size: int
    align: int
    fields: List[Field]

    def field_index(self, name: str) -> int:
        for i, f in enumerate(self.fields):
            if f.name == name:
                return i
        raise KeyError(name)


@dataclass
class Schema:
    types: List[Type]
    root_type: int = 0

    def type_index(self, name: str) -> int:
        for i, t in enumerate(self.types):
            if t.name == name:
                return i
        raise KeyError(name)


def to_ctypes(schema: Schema, field_cls, type_cls, schema_cls, field_args):
    """Lay a Schema out in some library's mirror structs.  Returns (struct, keepalive)."""
    keep = []
    types = (type_cls * len(schema.types))()
    for ti, t in enumerate(schema.types):
        fs = (field_cls * max(1, len(t.fields)))()
        for fi, f in enumerate(t.fields):
            for k, v in field_args(f).items():
                setattr(fs[fi], k, v)
        keep.append(fs)
        types[ti].size, types[ti].align, types[ti].nfields = t.size, t.align, len(t.fields)
        types[ti].fields = ctypes.cast(fs, ctypes.POINTER(field_cls))
    keep.append(types)
    s = schema_cls()
    s.ntypes, s.root_type = len(schema.types), schema.root_type
    s.types = ctypes.cast(types, ctypes.POINTER(type_cls))
    return s, keep


def _tg_field_args(f: Field):
    return dict(kind=f.kind, offset=f.offset, elem_size=f.elem_size, count_field=f.count_field,
                count_const=f.count_const, child_type=f.child_type, elem_kind=f.elem_kind)


# ---------------------------------------------------------------------------
# schemas used by the workloads
# ---------------------------------------------------------------------------

def node_schema() -> Schema:
    """``struct Node {int32 n; int32 nchild; float* position; float* velocity;
    Node* child;}`` — 32 bytes; ``nchild`` occupies the padding after ``n``."""
    return Schema([Type("Node", 32, 8, [
        Field("n", SCALAR, 0, 4),
        Field("nchild", SCALAR, 4, 4),
        Field("position", ARRAY, 8, 4, count_field=0, elem_kind=F32),
        Field("velocity", ARRAY, 16, 4, count_field=0, elem_kind=F32),
        Field("child", CHILD, 24, count_field=1, child_type=0),
    ])])


def linear_schema() -> Schema:
    """The Linear scenario's level struct (Fig 3): ``{int nA; int nLnext;
    double* A; L* Lnext}``, 24 bytes, chained through ``Lnext``."""
    return Schema([Type("L", 24, 8, [
        Field("nA", SCALAR, 0, 4),
        Field("nLnext", SCALAR, 4, 4),
        Field("A", ARRAY, 8, 8, count_field=0, elem_kind=F64),
        Field("Lnext", CHILD, 16, count_field=1, child_type=0),
    ])])


def dense_schema(D: int) -> Schema:
    """The Dense scenario (Fig 4): levels L0..L(D-1) are ``{int nA; int nLnext;
    double* A; L* Lnext}`` whose ``Lnext`` points to an array of q structs of the
    next level; the last level L(D) is the half-size ``{int nA; double* A}``
    (16 bytes with its padding)."""
    types = []
    for i in range(D):
        types.append(Type(f"L{i}", 24, 8, [
            Field("nA", SCALAR, 0, 4),
            Field("nLnext", SCALAR, 4, 4),
            Field("A", ARRAY, 8, 8, count_field=0, elem_kind=F64),
            Field("Lnext", CHILD, 16, count_field=1, child_type=i + 1),
        ]))
    types.append(Type(f"L{D}", 16, 8, [
        Field("nA", SCALAR, 0, 4),
        Field("A", ARRAY, 8, 8, count_field=0, elem_kind=F64),
    ]))
    return Schema(types)


def listing1_schema() -> Schema:
    """The three-type chain of Listing 1: Simulation -> Atoms -> Traits, whose
    ``double* positions[3]`` are three ARRAY fields of nAtoms doubles.  Each
    struct carries an extra scalar so the copied bytes include non-pointer data."""
    return Schema([
        Type("Simulation", 16, 8, [
            Field("step", SCALAR, 0, 8),
            Field("atoms", CHILD, 8, count_const=1, child_type=1),
        ]),
        Type("Atoms", 16, 8, [
            Field("nAtoms", SCALAR, 0, 4),
            Field("traits", CHILD, 8, count_const=1, child_type=2),
        ]),
        Type("Traits", 32, 8, [
            Field("n", SCALAR, 0, 4),
            Field("positions0", ARRAY, 8, 8, count_field=0, elem_kind=F64),
            Field("positions1", ARRAY, 16, 8, count_field=0, elem_kind=F64),
            Field("positions2", ARRAY, 24, 8, count_field=0, elem_kind=F64),
        ]),
    ])


# ---------------------------------------------------------------------------
# trees
# ---------------------------------------------------------------------------

@dataclass
class Rule:
    type: int
    field: int
    interior: tuple
    leaf: tuple


def const(v):
    return (CONST, float(v), 0.0, 0.0)


def uniform(lo, hi):
    return (UNIFORM, float(lo), float(hi), 0.0)


def lognormal(median, sigma, cap):
    return (LOGNORMAL, float(median), float(sigma), float(cap))


def _shape(levels: int, rules: Sequence[Rule], nthreads: int = 0):
    rs = (_Rule * max(1, len(rules)))()
    for i, r in enumerate(rules):
        rs[i].type, rs[i].field = r.type, r.field
        for dst, src in ((rs[i].interior, r.interior), (rs[i].leaf, r.leaf)):
            dst.dist, dst.a, dst.b, dst.c = src
    sh = _Shape()
    sh.levels, sh.nrules, sh.rules, sh.nthreads = levels, len(rules), rs, nthreads
    return sh, rs


class Tree:
    """One generated host tree.  ``root`` is the host address of the root struct.
    The memory is freed by ``free()`` (or when the object is collected)."""

    def __init__(self, schema: Schema, levels: int, rules: Sequence[Rule], seed: int,
                 name: str = "", nthreads: int = 0, alloc=None):
        """``alloc``: optional (function address, context) of a C allocator
        ``void* fn(void* ctx, uint64_t bytes, uint64_t align)`` that provides
        every block (e.g. an arena); such blocks are not freed by ``free()``."""
        L = lib()
        self.schema, self.levels, self.rules, self.seed, self.name = schema, levels, list(rules), seed, name
        cs, self._keep = to_ctypes(schema, _Field, _Type, _Schema, _tg_field_args)
        sh, rk = _shape(levels, rules, nthreads)
        self._keep.append(rk)
        if alloc is None:
            h = L.tg_build(ctypes.byref(cs), ctypes.byref(sh), seed)
        else:
            h = L.tg_build_ex(ctypes.byref(cs), ctypes.byref(sh), seed, alloc[0], alloc[1])
        if not h:
            raise RuntimeError("treegen: " + L.tg_error().decode())
        self._h = h
        self.root = L.tg_root(h)
        self.payload_bytes = L.tg_payload_bytes(h)
        self.nstructs = L.tg_nstructs(h)
        self.nblocks = L.tg_nblocks(h)

    def nelems(self, type_name: str, field_name: str) -> int:
        t = self.schema.type_index(type_name)
        f = self.schema.types[t].field_index(field_name)
        return lib().tg_nelems(self._h, t, f)

    def free(self):
        if getattr(self, "_h", None):
            lib().tg_free(self._h)
            self._h = None
            self.root = 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def dry_bytes(schema: Schema, levels: int, rules: Sequence[Rule], seed: int) -> int:
    cs, keep = to_ctypes(schema, _Field, _Type, _Schema, _tg_field_args)
    sh, rk = _shape(levels, rules)
    out = ctypes.c_uint64()
    if lib().tg_dry_bytes(ctypes.byref(cs), ctypes.byref(sh), seed, ctypes.byref(out)):
        raise RuntimeError("treegen: " + lib().tg_error().decode())
    return out.value


def node_tree(levels: int, fanout, n_interior, n_leaf=None, seed: int = 0, name: str = "",
              nthreads: int = 0, alloc=None) -> Tree:
    """A node-struct tree: ``fanout`` and the lengths are (dist, a, b, c) tuples
    or plain integers (constants)."""
    s = node_schema()
    f = fanout if isinstance(fanout, tuple) else const(fanout)
    ni = n_interior if isinstance(n_interior, tuple) else const(n_interior)
    nl = ni if n_leaf is None else (n_leaf if isinstance(n_leaf, tuple) else const(n_leaf))
    rules = [Rule(0, 0, ni, nl), Rule(0, 1, f, const(0))]
    return Tree(s, levels, rules, seed, name=name, nthreads=nthreads, alloc=alloc)


def linear_tree(k: int, n: int, layout: str = "allinit", seed: int = 0, alloc=None) -> Tree:
    """The Linear scenario with k levels and n doubles per A array.  ``allinit``
    allocates every level's A (allinit-allused / allinit-LLused); ``llinit``
    only the last level's (LLinit-LLused: the others are NULL, nA = 0)."""
    s = linear_schema()
    interior = const(n) if layout == "allinit" else const(0)
    rules = [Rule(0, 0, interior, const(n)), Rule(0, 1, const(1), const(0))]
    return Tree(s, k, rules, seed, name=f"linear-{layout}-k{k}-n{n}", alloc=alloc)


def dense_tree(q: int, n: int, D: int, seed: int = 0, alloc=None) -> Tree:
    """The Dense scenario: D+1 struct levels, q structs per intermediate array,
    n doubles per A array."""
    s = dense_schema(D)
    rules = []
    for i in range(D):
        rules.append(Rule(i, 0, const(n), const(n)))
        rules.append(Rule(i, 1, const(q), const(q)))
    rules.append(Rule(D, 0, const(n), const(n)))
    return Tree(s, D + 1, rules, seed, name=f"dense-q{q}-n{n}-D{D}", alloc=alloc)


def listing1_tree(n_atoms: int, seed: int = 0) -> Tree:
    s = listing1_schema()
    rules = [Rule(2, 0, const(n_atoms), const(n_atoms))]
    return Tree(s, 3, rules, seed, name=f"listing1-{n_atoms}")


# Named workloads ------------------------------------------------------------

WORKLOADS = {
    # name: (levels, fanout, n_interior, n_leaf, seed)
    "tiny": (4, 1, 65536, None, 1),
    "dense": (3, 16, lognormal(65536, 1.2, 4194304), None, 2),
    "deep": (64, 1, 1024, 1 << 26, 3),
    "reloc_stress": (6, 16, 10, None, 6),
}


def workload(name: str, seed: Optional[int] = None, nthreads: int = 0, alloc=None) -> Tree:
    levels, fanout, ni, nl, s = WORKLOADS[name]
    return node_tree(levels, fanout, ni, nl, seed=s if seed is None else seed, name=name,
                     nthreads=nthreads, alloc=alloc)


def leaf_path(levels: int, index: int = 0, child_field: int = 4):
    """The chain root->child[index]->...->child[index] down to the last level
    of a node tree, as (field, index) steps."""
    return [(child_field, index)] * (levels - 1)


# Random schemas for property tests -------------------------------------------

def random_schema(rng) -> tuple:
    """A random schema of 1-4 struct types with scalars, arrays (f32/f64/bytes,
    counted or constant) and child arrays, plus generation rules.  ``rng`` is a
    ``random.Random``.  Returns (schema, levels, rules)."""
    ntypes = rng.randint(1, 4)
    types = []
    rules = []
    for ti in range(ntypes):
        fields: List[Field] = []
        off = 0
        nscal = rng.randint(1, 3)
        for si in range(nscal):
            w = rng.choice([4, 8])
            off = (off + w - 1) // w * w
            fields.append(Field(f"s{si}", SCALAR, off, w))
            off += w
        npt = rng.randint(0, 4)
        nchild = 0
        for pi in range(npt):
            off = (off + 7) // 8 * 8
            kind = rng.choice([ARRAY, ARRAY, CHILD]) if nchild < 2 else ARRAY
            nchild += kind == CHILD
            cf = rng.randrange(nscal)
            if kind == ARRAY:
                ek = rng.choice([F32, F64, BYTES])
                es = {F32: 4, F64: 8, BYTES: rng.choice([1, 2, 3, 12])}[ek]
                if rng.random() < 0.2:
                    fields.append(Field(f"a{pi}", ARRAY, off, es, count_const=rng.randint(0, 9),
                                        elem_kind=ek))
                else:
                    fields.append(Field(f"a{pi}", ARRAY, off, es, count_field=cf, elem_kind=ek))
            else:
                fields.append(Field(f"c{pi}", CHILD, off, count_field=cf,
                                    child_type=rng.randrange(ntypes)))
            off += 8
        off += rng.choice([0, 4, 8])
        size = max(8, (off + 7) // 8 * 8)
        types.append(Type(f"T{ti}", size, 8, fields))
        for si in range(nscal):
            rules.append(Rule(ti, si, uniform(0, rng.choice([0, 1, 2, 3])),
                              uniform(0, rng.choice([0, 7, 33, 5000]))))
    levels = rng.randint(1, 6)
    return Schema(types, rng.randrange(ntypes)), levels, rules


# Batched workload ------------------------------------------------------------------

def poisson_requests(duration: float, rate: float = 2000.0, retouch: float = 0.3, seed: int = 5):
    """A request stream: arrivals of a Poisson process of ``rate`` per second
    over ``duration`` seconds; each request re-touches a key served before
    (uniform over them) with probability ``retouch``, else names a new key.
    Returns ([(key, arrival_s, retouch 0/1)], number of keys)."""
    import random as _random
    rng = _random.Random(seed)
    reqs, nkeys, t = [], 0, 0.0
    while True:
        t += rng.expovariate(rate)
        if t >= duration:
            break
        if nkeys and rng.random() < retouch:
            reqs.append((rng.randrange(nkeys), t, 1))
        else:
            reqs.append((nkeys, t, 0))
            nkeys += 1
    return reqs, nkeys


@dataclass
class TreeSpec:
    """One tree of the batched workload before it is built: its shape, its
    seed and its payload bytes (counted without allocating)."""
    levels: int
    rules: List[Rule]
    seed: int
    bytes: int
    index: int

    def build(self, name: str = "") -> Tree:
        return Tree(node_schema(), self.levels, self.rules, self.seed, name=name or f"batched-{self.index}",
                    nthreads=1)


def batched_specs(ntrees: int = 4096, seed: int = 4, t_min: int = 16 << 10, t_max: int = 7 << 20,
                  median: int = 4096, sigma: float = 1.0, cap: int = 1 << 20) -> List[TreeSpec]:
    """The shapes of ``batched(...)``'s trees, drawn the same way, without
    building them: per tree, levels uniform in 1-5 and fanout uniform in 1-8;
    array lengths lognormal (median ``median``, sigma ``sigma``, capped at
    ``cap``); a tree whose payload falls outside [t_min, t_max] bytes is
    redrawn with the next seed.  The first k specs of a longer draw are the
    specs of a draw of k."""
    import random as _random
    rng = _random.Random(seed)
    specs = []
    for i in range(ntrees):
        while True:
            levels, fanout, s = rng.randint(1, 5), rng.randint(1, 8), rng.getrandbits(63)
            n = lognormal(median, sigma, cap)
            rules = [Rule(0, 0, n, n), Rule(0, 1, const(fanout), const(0))]
            b = dry_bytes(node_schema(), levels, rules, s)
            if t_min <= b <= t_max:
                break
        specs.append(TreeSpec(levels, rules, s, b, i))
    return specs


def batched(ntrees: int = 4096, seed: int = 4, t_min: int = 16 << 10, t_max: int = 7 << 20,
            median: int = 4096, sigma: float = 1.0, cap: int = 1 << 20):
    """``ntrees`` independent node trees of uneven shape (``batched_specs``),
    built."""
    return [sp.build() for sp in batched_specs(ntrees, seed, t_min, t_max, median, sigma, cap)]


# Address-only trees ----------------------------------------------------------------

class ReservedChain:
    """A Linear chain (``linear_schema``) of ``levels`` level structs whose A
    arrays are address ranges reserved with no memory behind them
    (``mmap(PROT_NONE, MAP_NORESERVE)``), each ``nA`` doubles long.  Planning
    reads only the level structs, so such a tree lays out an arena far larger
    than the host's memory (at nA = 2^31 - 2, 16 GiB per level) without
    touching the arrays; it is for layout and relocation tests only: reading
    an A array faults.  ``root`` is the level-0 struct's address."""

    PROT_NONE, MAP_PRIVATE, MAP_ANONYMOUS, MAP_NORESERVE = 0, 0x02, 0x20, 0x4000

    def __init__(self, levels: int, nA: int):
        libc = ctypes.CDLL(None, use_errno=True)
        libc.mmap.restype = ctypes.c_void_p
        libc.mmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.c_long]
        libc.munmap.restype = ctypes.c_int
        libc.munmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
        self._libc, self.schema, self.levels, self.nA, self.name = libc, linear_schema(), levels, nA, "reserved"
        self.span = (nA * 8 + 4095) // 4096 * 4096
        self.region = libc.mmap(None, self.span * levels, self.PROT_NONE,
                                self.MAP_PRIVATE | self.MAP_ANONYMOUS | self.MAP_NORESERVE, -1, 0)
        if self.region in (None, ctypes.c_void_p(-1).value):
            raise OSError(ctypes.get_errno(), "mmap of the reserved A arrays failed")

        class L(ctypes.Structure):
            _fields_ = [("nA", ctypes.c_int32), ("nLnext", ctypes.c_int32), ("A", ctypes.c_void_p),
                        ("Lnext", ctypes.c_void_p)]

        # one single-struct array per level (Lnext has count 1), the last with no next level
        self.levels_c = [L() for _ in range(levels)]
        for k, s in enumerate(self.levels_c):
            s.nA, s.A = nA, self.region + k * self.span
            if k + 1 < levels:
                s.nLnext, s.Lnext = 1, ctypes.addressof(self.levels_c[k + 1])
        self.root = ctypes.addressof(self.levels_c[0])

    def free(self):
        if getattr(self, "region", None):
            self._libc.munmap(self.region, self.span * self.levels)
            self.region, self.root = None, 0

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
