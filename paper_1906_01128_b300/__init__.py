"""Python binding of ``libdc.so``, the B300 deep-copy library (C ABI in
``include/dc.h``).

Argument marshalling only: every step of the deep-copy path runs in the
library's C++ runtime and CUDA kernels.  PyTorch provides device memory (the
arena a plan is bound to is a ``torch.uint8`` CUDA tensor) and streams.  There
is no fallback: importing this package fails if the library is not built.

Typical flow (Algorithm 2: transfer, run the kernel once, transfer back)::

    plan = Plan(schema, host_root)        # walk + layout (Algorithm 1 step 1)
    plan.bind()                           # device arena from torch
    plan.deep_copy()                      # marshal, H2D, relocate (Fig 2 b-d)
    plan.update(Op())                     # leaf kernel through resolved chains
    plan.copy_back()                      # results back into the host arrays
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import torch  # loads the CUDA runtime that libdc.so then shares

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdc.so")

OP_AXPY_HALF, OP_SCALE = 0, 1
SEL_ALL, SEL_CHAIN = 0, 1
PLAN_VERIFY = 1
PLAN_MAP_HOST = 2
PLAN_DEVICE_SCAN = 4
PLAN_PACK_SMALL = 8
PLAN_SPANS = 16
COPY_ALL_ARRAYS = 1

STATUS = {0: "DC_OK", 1: "DC_EINVAL", 2: "DC_ENOMEM", 3: "DC_ECUDA", 4: "DC_EALIAS", 5: "DC_ECYCLE",
          6: "DC_EBUDGET", 7: "DC_ETIMEOUT", 8: "DC_EDEVICE_BOUNDS", 9: "DC_ESTATE", 10: "DC_EVERIFY"}


class DcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class _Field(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("offset", ctypes.c_uint32), ("elem_size", ctypes.c_uint32),
                ("count_field", ctypes.c_int32), ("count_const", ctypes.c_uint64),
                ("child_type", ctypes.c_int32), ("elem_kind", ctypes.c_int32)]


class _Type(ctypes.Structure):
    _fields_ = [("size", ctypes.c_uint32), ("align", ctypes.c_uint32), ("nfields", ctypes.c_uint32),
                ("fields", ctypes.POINTER(_Field))]


class _Schema(ctypes.Structure):
    _fields_ = [("ntypes", ctypes.c_uint32), ("root_type", ctypes.c_uint32),
                ("types", ctypes.POINTER(_Type))]


class _Step(ctypes.Structure):
    _fields_ = [("field", ctypes.c_uint32), ("index", ctypes.c_uint64)]


class _Op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("scale", ctypes.c_double), ("sel", ctypes.c_int32),
                ("path", ctypes.POINTER(_Step)), ("path_len", ctypes.c_uint32), ("type", ctypes.c_uint32),
                ("x_field", ctypes.c_uint32), ("y_field", ctypes.c_uint32)]


class _Info(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("data_bytes", "device_bytes", "payload_bytes", "nblocks",
                                               "nrelocs", "nstructs", "nstruct_blocks", "root_offset",
                                               "ntrees", "struct_bytes", "reloc_table_bytes",
                                               "staging_bytes")]


class _Request(ctypes.Structure):
    _fields_ = [("key", ctypes.c_uint64), ("host_root", ctypes.c_void_p), ("arrival_s", ctypes.c_double),
                ("retouch", ctypes.c_int32)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("served", "failed", "resident_hits", "evictions", "h2d_bytes",
                                               "d2h_bytes", "peak_resident_bytes", "resident_bytes")] + \
               [("wall_s", ctypes.c_double)]


# every entry point of include/dc.h, with its argument types
_P = ctypes.POINTER
_vp, _u32, _u64, _i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
SIGNATURES = {
    "dc_plan": [_P(_Schema), _vp, _P(_vp)],
    "dc_plan_forest": [_P(_Schema), _P(_vp), _u64, _P(_vp)],
    "dc_plan_root": [_vp, _u64, _P(_u64)],
    "dc_plan_set_flags": [_vp, _u32],
    "dc_plan_info_get": [_vp, _P(_Info)],
    "dc_plan_arena_bytes": [_vp, _P(_u64), _P(_u64), _P(_u64)],
    "dc_plan_block": [_vp, _u64, _P(_u64), _P(_u64), _P(_u64), _P(_u32), _P(_u32), _P(_u32)],
    "dc_plan_set_threads": [_vp, _u32],
    "dc_plan_destroy": [_vp],
    "dc_bind_device": [_vp, _vp, _u64, _vp],
    "dc_deep_copy": [_vp, _vp],
    "dc_deep_copy_selected": [_vp, _P(_Op), _vp],
    "dc_relocate": [_vp, _vp],
    "dc_relocate_static": [_vp, _vp, _u64, _vp, _vp],
    "dc_resolve_chain": [_vp, _P(_Step), _u32, _P(_u64)],
    "dc_resolve_offset": [_vp, _P(_Step), _u32, _P(_u64)],
    "dc_resolve_chain_in": [_vp, _u64, _P(_Step), _u32, _P(_u64)],
    "dc_resolve_offset_in": [_vp, _u64, _P(_Step), _u32, _P(_u64)],
    "dc_relocate_update": [_vp, _P(_Op), _vp],
    "dc_autotune": [_vp, _P(_Op), _vp, _P(_u32), _P(_u32)],
    "dc_set_split": [_vp, _P(_Op), _u32, _u32],
    "dc_partition_by_bytes": [_P(_u64), _u64, _u32, _P(_u32), _P(_u64)],
    "dc_update_leaves": [_vp, _P(_Op), _vp],
    "dc_update_chase": [_vp, _P(_Op), _vp],
    "dc_verify_chain": [_vp, _P(_Step), _u32, _vp, _P(_u64)],
    "dc_copy_back": [_vp, _u32, _vp],
    "dc_roundtrip": [_vp, _P(_Op), _vp],
    "dc_roundtrip_selected": [_vp, _P(_Op), _vp],
    "dc_sync": [_vp, _vp],
    "dc_device_base": [_vp, _P(_u64)],
    "dc_uvm_build": [_P(_Schema), _vp, _P(_vp)],
    "dc_uvm_root": [_vp, _P(_u64)],
    "dc_uvm_prefetch": [_vp, _i32, _vp],
    "dc_uvm_update": [_vp, _P(_Op), _vp],
    "dc_uvm_copy_back": [_vp, _vp, _u32],
    "dc_uvm_sync": [_vp, _vp],
    "dc_uvm_destroy": [_vp],
    "dc_server_create": [_P(_Schema), _vp, _u64, _u64, _u32, _u32, _P(_vp)],
    "dc_server_run": [_vp, _P(_Request), _u64, _P(_Op), _P(ctypes.c_double)],
    "dc_server_stats_get": [_vp, _P(_ServerStats)],
    "dc_server_destroy": [_vp],
    "dc_host_arena_create": [_u64, _P(_vp)],
    "dc_host_arena_used": [_vp, _P(_u64)],
    "dc_host_arena_reset": [_vp],
    "dc_host_arena_destroy": [_vp],
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libdc.so is not built ({LIB_PATH}); run paper_1906_01128_b300/build.py "
                          "or __graft_entry__.build() — there is no fallback implementation")
    L = ctypes.CDLL(LIB_PATH)
    for name, args in SIGNATURES.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.dc_last_error.restype = ctypes.c_char_p
    L.dc_last_error.argtypes = []
    L.dc_status_name.restype = ctypes.c_char_p
    L.dc_status_name.argtypes = [ctypes.c_int]
    L.dc_kernel_launches.restype = ctypes.c_uint64
    L.dc_kernel_launches.argtypes = []
    L.dc_host_arena_alloc.restype = ctypes.c_void_p
    L.dc_host_arena_alloc.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64]
    return L


lib = _load()


def _check(status: int):
    if status != 0:
        raise DcError(status, lib.dc_last_error().decode(errors="replace"))


def kernel_launches() -> int:
    """Kernels this library has launched in this process."""
    return lib.dc_kernel_launches()


def partition_by_bytes(sizes: Sequence[int], nparts: int) -> Tuple[List[int], List[int]]:
    """dc_partition_by_bytes: (part of each tree, bytes of each part), greedy LPT."""
    n = len(sizes)
    b = (ctypes.c_uint64 * max(n, 1))(*sizes)
    part = (ctypes.c_uint32 * max(n, 1))()
    load = (ctypes.c_uint64 * max(nparts, 1))()
    _check(lib.dc_partition_by_bytes(b, n, nparts, part, load))
    return list(part[:n]), list(load[:nparts])


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def schema_struct(schema):
    """ctypes ``dc_schema`` for any object with ``types`` (each with size, align,
    fields) and ``root_type``; returns (struct, keepalive)."""
    keep = []
    types = (_Type * len(schema.types))()
    for ti, t in enumerate(schema.types):
        fs = (_Field * max(1, len(t.fields)))()
        for fi, f in enumerate(t.fields):
            fs[fi] = _Field(f.kind, f.offset, f.elem_size, f.count_field, f.count_const, f.child_type,
                            f.elem_kind)
        keep.append(fs)
        types[ti] = _Type(t.size, t.align, len(t.fields), ctypes.cast(fs, ctypes.POINTER(_Field)))
    keep.append(types)
    return _Schema(len(schema.types), schema.root_type, ctypes.cast(types, ctypes.POINTER(_Type))), keep


def _steps(path: Sequence[Tuple[int, int]]):
    arr = (_Step * max(1, len(path)))()
    for i, (f, ix) in enumerate(path):
        arr[i] = _Step(f, ix)
    return arr


@dataclass
class Op:
    """A leaf-kernel request (``dc_op``): kind OP_AXPY_HALF (x += 0.5*y) or
    OP_SCALE (x *= scale); sel SEL_ALL (every struct of ``type``) or SEL_CHAIN
    (the struct ``path`` reaches, as (child field, index) steps)."""
    kind: int = OP_AXPY_HALF
    sel: int = SEL_ALL
    type: int = 0
    x_field: int = 2
    y_field: int = 3
    scale: float = 1.0
    path: Sequence[Tuple[int, int]] = ()


def _op(op):
    steps = _steps(op.path)
    o = _Op(op.kind, op.scale, op.sel, ctypes.cast(steps, ctypes.POINTER(_Step)), len(op.path), op.type,
            op.x_field, op.y_field)
    return o, steps


class Plan:
    """``dc_plan_t``: the walk and layout of one host tree, then its device copy."""

    def __init__(self, schema, host_root, flags: int = 0, threads: int = 0):
        """``host_root``: the root's address, or a sequence of root addresses
        for a forest (``dc_plan_forest``)."""
        self._schema_c, self._keep = schema_struct(schema)
        h = ctypes.c_void_p()
        if isinstance(host_root, int):
            _check(lib.dc_plan(ctypes.byref(self._schema_c), host_root, ctypes.byref(h)))
        else:
            roots = (ctypes.c_void_p * len(host_root))(*host_root)
            _check(lib.dc_plan_forest(ctypes.byref(self._schema_c), roots, len(host_root), ctypes.byref(h)))
        self._h = h.value
        self.host_root = host_root if isinstance(host_root, int) else host_root[0]
        self.flags = flags
        if flags:
            _check(lib.dc_plan_set_flags(self._h, flags))
        if threads:
            _check(lib.dc_plan_set_threads(self._h, threads))
        self.buffer: Optional[torch.Tensor] = None

    def arena_bytes(self) -> tuple:
        """(device buffer bytes for bind, blocks, pointer slots) — dc_plan_arena_bytes."""
        b, n, r = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib.dc_plan_arena_bytes(self._h, ctypes.byref(b), ctypes.byref(n), ctypes.byref(r)))
        return b.value, n.value, r.value

    @property
    def info(self) -> dict:
        i = _Info()
        _check(lib.dc_plan_info_get(self._h, ctypes.byref(i)))
        return {n: getattr(i, n) for n, _ in _Info._fields_}

    def block(self, i: int) -> dict:
        h, o, b = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        l, par, so = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib.dc_plan_block(self._h, i, ctypes.byref(h), ctypes.byref(o), ctypes.byref(b), ctypes.byref(l),
                                 ctypes.byref(par), ctypes.byref(so)))
        return dict(host=h.value, offset=o.value, bytes=b.value, lane=l.value,
                    parent=None if par.value == 0xFFFFFFFF else par.value, slot_off=so.value)

    def blocks(self):
        return [self.block(i) for i in range(self.info["nblocks"])]

    def set_threads(self, n: int):
        _check(lib.dc_plan_set_threads(self._h, n))

    def set_flags(self, flags: int):
        """dc_plan_set_flags (DC_PLAN_PACK_SMALL lays the plan out again)."""
        _check(lib.dc_plan_set_flags(self._h, flags))
        self.flags = flags

    def bind(self, buffer: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        need = self.info["device_bytes"]
        if buffer is None:
            buffer = torch.empty(need, dtype=torch.uint8, device="cuda")
        _check(lib.dc_bind_device(self._h, buffer.data_ptr(), buffer.numel() * buffer.element_size(),
                                  _stream(stream)))
        self.buffer = buffer
        return buffer

    def deep_copy(self, stream=None):
        _check(lib.dc_deep_copy(self._h, _stream(stream)))

    def deep_copy_selected(self, op=None, stream=None):
        """Selective deep copy: the struct blocks on the op's chain(s) and its arrays."""
        o, keep = _op(op or Op())
        _check(lib.dc_deep_copy_selected(self._h, ctypes.byref(o), _stream(stream)))

    def relocate(self, stream=None):
        _check(lib.dc_relocate(self._h, _stream(stream)))

    def resolve(self, path) -> int:
        st, out = _steps(path), ctypes.c_uint64()
        _check(lib.dc_resolve_chain(self._h, st, len(path), ctypes.byref(out)))
        return out.value

    def root_offset(self, tree: int) -> int:
        out = ctypes.c_uint64()
        _check(lib.dc_plan_root(self._h, tree, ctypes.byref(out)))
        return out.value

    def resolve_in(self, tree: int, path) -> int:
        st, out = _steps(path), ctypes.c_uint64()
        _check(lib.dc_resolve_chain_in(self._h, tree, st, len(path), ctypes.byref(out)))
        return out.value

    def relocate_update(self, op=None, stream=None):
        """dc_relocate + dc_update_leaves in one persistent launch."""
        o, keep = _op(op or Op())
        _check(lib.dc_relocate_update(self._h, ctypes.byref(o), _stream(stream)))

    def autotune(self, op=None, stream=None):
        """Pick the fused launch's split; returns (threads per CTA, CTAs per SM)."""
        o, keep = _op(op or Op())
        t, c = ctypes.c_uint32(), ctypes.c_uint32()
        _check(lib.dc_autotune(self._h, ctypes.byref(o), _stream(stream), ctypes.byref(t), ctypes.byref(c)))
        return t.value, c.value

    def set_split(self, op=None, threads: int = 256, ctas_per_sm: int = 0):
        """Pin the fused launch's split (dc_set_split) instead of timing candidates."""
        o, keep = _op(op or Op())
        _check(lib.dc_set_split(self._h, ctypes.byref(o), threads, ctas_per_sm))

    def resolve_offset(self, path) -> int:
        st, out = _steps(path), ctypes.c_uint64()
        _check(lib.dc_resolve_offset(self._h, st, len(path), ctypes.byref(out)))
        return out.value

    def verify_chain(self, path, stream=None) -> int:
        st, out = _steps(path), ctypes.c_uint64()
        _check(lib.dc_verify_chain(self._h, st, len(path), _stream(stream), ctypes.byref(out)))
        return out.value

    def update(self, op=None, stream=None):
        o, keep = _op(op or Op())
        _check(lib.dc_update_leaves(self._h, ctypes.byref(o), _stream(stream)))

    def update_chase(self, op=None, stream=None):
        o, keep = _op(op or Op())
        _check(lib.dc_update_chase(self._h, ctypes.byref(o), _stream(stream)))

    def roundtrip(self, op=None, stream=None):
        """deep_copy + update(op) + copy_back in one pipelined call."""
        o, keep = _op(op or Op())
        _check(lib.dc_roundtrip(self._h, ctypes.byref(o), _stream(stream)))

    def roundtrip_selected(self, op=None, stream=None):
        """Move only the op's arrays (pointerchain), update, copy x back."""
        o, keep = _op(op or Op())
        _check(lib.dc_roundtrip_selected(self._h, ctypes.byref(o), _stream(stream)))

    def copy_back(self, all_arrays: bool = False, stream=None):
        _check(lib.dc_copy_back(self._h, COPY_ALL_ARRAYS if all_arrays else 0, _stream(stream)))

    def sync(self, stream=None):
        _check(lib.dc_sync(self._h, _stream(stream)))

    @property
    def device_base(self) -> int:
        out = ctypes.c_uint64()
        _check(lib.dc_device_base(self._h, ctypes.byref(out)))
        return out.value

    def image(self):
        """A host (numpy) copy of the device arena's data region."""
        n = self.info["data_bytes"]
        torch.cuda.synchronize()
        return self.buffer[:n].cpu().numpy()

    def destroy(self):
        if getattr(self, "_h", None):
            lib.dc_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Uvm:
    """``dc_uvm_t``: a managed-memory replica of a host tree (comparison path)."""

    def __init__(self, schema, host_root: int):
        self._schema_c, self._keep = schema_struct(schema)
        h = ctypes.c_void_p()
        _check(lib.dc_uvm_build(ctypes.byref(self._schema_c), host_root, ctypes.byref(h)))
        self._h = h.value
        self.host_root = host_root

    @property
    def root(self) -> int:
        out = ctypes.c_uint64()
        _check(lib.dc_uvm_root(self._h, ctypes.byref(out)))
        return out.value

    def prefetch(self, to_device: bool, stream=None):
        _check(lib.dc_uvm_prefetch(self._h, 1 if to_device else 0, _stream(stream)))

    def update(self, op=None, stream=None):
        o, keep = _op(op or Op())
        _check(lib.dc_uvm_update(self._h, ctypes.byref(o), _stream(stream)))

    def sync(self, stream=None):
        _check(lib.dc_uvm_sync(self._h, _stream(stream)))

    def copy_back(self, all_arrays: bool = False):
        _check(lib.dc_uvm_copy_back(self._h, self.host_root, COPY_ALL_ARRAYS if all_arrays else 0))

    def destroy(self):
        if getattr(self, "_h", None):
            lib.dc_uvm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


SERVER_SEQUENTIAL = 1


class Server:
    """``dc_server_t``: a request loop over a device pool (a torch CUDA uint8
    tensor, the HBM budget) with ``slots`` concurrent workers."""

    def __init__(self, schema, pool: torch.Tensor, pinned_bytes: int, slots: int = 4, flags: int = 0):
        self._schema_c, self._keep = schema_struct(schema)
        h = ctypes.c_void_p()
        _check(lib.dc_server_create(ctypes.byref(self._schema_c), pool.data_ptr(), pool.numel(), pinned_bytes,
                                    slots, flags, ctypes.byref(h)))
        self._h = h.value
        self.pool = pool

    def run(self, requests, op=None):
        """requests: (key, host_root, arrival_s, retouch) tuples.  Returns the
        per-request latencies in ms (-1 for a failed request)."""
        n = len(requests)
        arr = (_Request * max(1, n))()
        for i, (k, r, a, t) in enumerate(requests):
            arr[i] = _Request(k, r, a, int(t))
        lat = (ctypes.c_double * max(1, n))()
        o, keep = _op(op or Op())
        _check(lib.dc_server_run(self._h, arr, n, ctypes.byref(o), lat))
        return list(lat)[:n]

    @property
    def stats(self) -> dict:
        st = _ServerStats()
        _check(lib.dc_server_stats_get(self._h, ctypes.byref(st)))
        return {n: getattr(st, n) for n, _ in _ServerStats._fields_}

    def destroy(self):
        if getattr(self, "_h", None):
            lib.dc_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class HostArena:
    """``dc_host_arena_t``: pinned, mapped host memory of the library's own to
    build trees in (Algorithm 1's allocation requests served from one
    buffer); plans move its blocks without a marshal.  ``allocator`` is the
    (function address, context) pair for C code that builds trees."""

    def __init__(self, nbytes: int):
        h = ctypes.c_void_p()
        _check(lib.dc_host_arena_create(nbytes, ctypes.byref(h)))
        self._h = h.value

    @property
    def allocator(self):
        return ctypes.cast(lib.dc_host_arena_alloc, ctypes.c_void_p).value, self._h

    def alloc(self, nbytes: int, align: int = 16) -> int:
        return lib.dc_host_arena_alloc(self._h, nbytes, align) or 0

    @property
    def used(self) -> int:
        out = ctypes.c_uint64()
        _check(lib.dc_host_arena_used(self._h, ctypes.byref(out)))
        return out.value

    def reset(self):
        _check(lib.dc_host_arena_reset(self._h))

    def destroy(self):
        if getattr(self, "_h", None):
            lib.dc_host_arena_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass
