"""CPU oracle for the deep-copy hot path — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It is plain C (``oracle.c``, built with
gcc, ``-ffp-contract=off``) behind ctypes, and shares no code with the CUDA
path; the two meet only in the seeded inputs of ``treegen``.

Each function follows a passage of the paper (see ``oracle.h``):
full deep copy (Sec. 2, Fig 2), the scaling / axpy leaf kernel (Sec. 4.1.2,
Listing 2), transfer back (Alg 2 step 5), the results check (Alg 2 step 6),
and effective-address extraction of a pointer chain (Sec. 3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

import numpy as np

import treegen as _tg

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")

OP_AXPY_HALF, OP_SCALE = 0, 1
SEL_ALL, SEL_CHAIN = 0, 1


def build_lib(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(hdr)):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-fno-fast-math", "-o", _SO, src])
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


class _Arena(ctypes.Structure):
    _fields_ = [("base", ctypes.c_void_p), ("cap", ctypes.c_uint64),
                ("used", ctypes.c_uint64), ("ptr_base", ctypes.c_uint64)]


class _Counts(ctypes.Structure):
    _fields_ = [("nstructs", ctypes.c_uint64), ("nblocks", ctypes.c_uint64),
                ("payload_bytes", ctypes.c_uint64), ("padded_bytes", ctypes.c_uint64),
                ("nptr", ctypes.c_uint64), ("levels", ctypes.c_uint32),
                ("per_level", ctypes.c_uint64 * 64)]


class _Step(ctypes.Structure):
    _fields_ = [("field", ctypes.c_uint32), ("index", ctypes.c_uint64)]


class _Op(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("scale", ctypes.c_double), ("sel", ctypes.c_int32),
                ("path", ctypes.POINTER(_Step)), ("path_len", ctypes.c_uint32),
                ("type", ctypes.c_uint32), ("x_field", ctypes.c_uint32),
                ("y_field", ctypes.c_uint32)]


_L = None


def lib():
    global _L
    if _L is None:
        L = ctypes.CDLL(build_lib())
        P = ctypes.POINTER
        L.or_count.argtypes = [P(_Schema), ctypes.c_void_p, P(_Counts)]
        L.or_deep_copy.argtypes = [P(_Schema), ctypes.c_void_p, P(_Arena), P(ctypes.c_void_p)]
        L.or_update.argtypes = [P(_Schema), ctypes.c_void_p, P(_Op)]
        L.or_update_parallel.argtypes = [P(_Schema), ctypes.c_void_p, P(_Op), ctypes.c_int]
        L.or_threads.argtypes = []
        L.or_copy_back.argtypes = [P(_Schema), ctypes.c_void_p, ctypes.c_void_p, P(_Op), ctypes.c_int]
        L.or_trees_equal.argtypes = [P(_Schema), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p,
                                     ctypes.c_size_t]
        L.or_check_image.argtypes = [P(_Schema), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                     ctypes.c_uint64, ctypes.c_uint64, P(_Counts), ctypes.c_char_p,
                                     ctypes.c_size_t]
        L.or_check_image_packed.argtypes = [P(_Schema), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, P(_Counts),
                                            ctypes.c_char_p, ctypes.c_size_t]
        L.or_check_chain_image.argtypes = [P(_Schema), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                           ctypes.c_uint64, ctypes.c_uint64, P(_Step), ctypes.c_uint32,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p, ctypes.c_size_t]
        L.or_image_resolve.argtypes = [P(_Schema), ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_uint64, P(_Step), ctypes.c_uint32,
                                       P(ctypes.c_uint64)]
        L.or_host_resolve.argtypes = [P(_Schema), ctypes.c_void_p, P(_Step), ctypes.c_uint32,
                                      P(ctypes.c_uint64)]
        for f in ("or_count", "or_deep_copy", "or_update", "or_update_parallel", "or_threads", "or_copy_back",
                  "or_trees_equal", "or_check_image", "or_check_image_packed", "or_check_chain_image", "or_image_resolve",
                  "or_host_resolve"):
            getattr(L, f).restype = ctypes.c_int
        _L = L
    return _L


def _field_args(f):
    return dict(kind=f.kind, offset=f.offset, elem_size=f.elem_size, count_field=f.count_field,
                count_const=f.count_const, child_type=f.child_type, elem_kind=f.elem_kind)


class _CSchema:
    """Cache of the ctypes mirror of a treegen.Schema."""

    def __init__(self, schema):
        self.struct, self._keep = _tg.to_ctypes(schema, _Field, _Type, _Schema, _field_args)


def _cs(schema) -> _CSchema:
    c = getattr(schema, "_oracle_c", None)
    if c is None:
        c = _CSchema(schema)
        schema._oracle_c = c
    return c


def _steps(path: Sequence[Tuple[int, int]]):
    arr = (_Step * max(1, len(path)))()
    for i, (f, ix) in enumerate(path):
        arr[i].field, arr[i].index = f, ix
    return arr


@dataclass
class Op:
    """A leaf-kernel request: ``kind`` OP_AXPY_HALF (x += 0.5*y) or OP_SCALE
    (x *= scale); ``sel`` SEL_ALL (every struct of ``type``) or SEL_CHAIN (the
    struct reached by ``path``, a list of (child field, index) steps)."""
    kind: int = OP_AXPY_HALF
    sel: int = SEL_ALL
    type: int = 0
    x_field: int = 2
    y_field: int = 3
    scale: float = 1.0
    path: Sequence[Tuple[int, int]] = ()


def _op(op: Op):
    steps = _steps(op.path)
    o = _Op(op.kind, op.scale, op.sel, ctypes.cast(steps, ctypes.POINTER(_Step)), len(op.path),
            op.type, op.x_field, op.y_field)
    return o, steps


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def count(schema, root: int) -> dict:
    c = _Counts()
    _check(lib().or_count(ctypes.byref(_cs(schema).struct), root, ctypes.byref(c)), "count")
    return _counts_dict(c)


def _counts_dict(c: _Counts) -> dict:
    return dict(nstructs=c.nstructs, nblocks=c.nblocks, payload_bytes=c.payload_bytes,
                padded_bytes=c.padded_bytes, nptr=c.nptr, levels=c.levels,
                per_level=[c.per_level[i] for i in range(min(c.levels, 64))])


class Copy:
    """An oracle deep copy: ``buf`` is the fresh arena (numpy uint8), ``root``
    the copied root's address.  With ``ptr_base`` the copied pointers are
    written relative to that base (an image of another address space)."""

    def __init__(self, schema, src_root: int, ptr_base: int = 0, extra: int = 0):
        need = count(schema, src_root)["padded_bytes"] + extra
        self.buf = np.zeros(max(16, need) + 16, dtype=np.uint8)
        addr = self.buf.ctypes.data
        pad = (-addr) % 16
        self.base = addr + pad
        self.cap = need
        a = _Arena(self.base, self.cap, 0, ptr_base)
        out = ctypes.c_void_p()
        _check(lib().or_deep_copy(ctypes.byref(_cs(schema).struct), src_root, ctypes.byref(a),
                                  ctypes.byref(out)), "deep_copy")
        self.used = a.used
        self.root = out.value
        self.schema = schema
        self.ptr_base = ptr_base

    def image(self) -> np.ndarray:
        off = self.base - self.buf.ctypes.data
        return self.buf[off:off + self.used]


def deep_copy(schema, src_root: int, ptr_base: int = 0) -> Copy:
    return Copy(schema, src_root, ptr_base)


def update(schema, root: int, op: Op) -> None:
    o, keep = _op(op)
    _check(lib().or_update(ctypes.byref(_cs(schema).struct), root, ctypes.byref(o)), "update")


def update_parallel(schema, root: int, op: Op, threads: int = 0) -> None:
    """``update`` on ``threads`` host cores (0 = all): the multi-core CPU baseline,
    bit-identical to ``update``."""
    o, keep = _op(op)
    _check(lib().or_update_parallel(ctypes.byref(_cs(schema).struct), root, ctypes.byref(o), threads),
           "update_parallel")


def threads() -> int:
    """Host threads ``update_parallel`` uses by default."""
    return lib().or_threads()


def copy_back(schema, copy_root: int, src_root: int, op: Optional[Op], all_arrays: bool = False):
    if op is None:
        rc = lib().or_copy_back(ctypes.byref(_cs(schema).struct), copy_root, src_root, None, 1)
    else:
        o, keep = _op(op)
        rc = lib().or_copy_back(ctypes.byref(_cs(schema).struct), copy_root, src_root,
                                ctypes.byref(o), int(all_arrays))
    _check(rc, "copy_back")


def trees_equal(schema, a: int, b: int) -> Tuple[bool, str]:
    msg = ctypes.create_string_buffer(1024)
    rc = lib().or_trees_equal(ctypes.byref(_cs(schema).struct), a, b, msg, 1024)
    if rc not in (0, 3):
        raise RuntimeError(f"oracle trees_equal: invalid tree (status {rc})")
    return rc == 0, msg.value.decode()


def check_image(schema, src_root: int, image: np.ndarray, dev_base: int, root_off: int = 0, pack_below: int = 0):
    """Check a host copy of a device arena's data region against the source tree.
    ``pack_below``: arrays of fewer bytes may start on their element alignment."""
    image = np.ascontiguousarray(image, dtype=np.uint8)
    msg = ctypes.create_string_buffer(1024)
    c = _Counts()
    rc = lib().or_check_image_packed(ctypes.byref(_cs(schema).struct), src_root, image.ctypes.data,
                                     image.nbytes, dev_base, root_off, pack_below, ctypes.byref(c), msg, 1024)
    if rc not in (0, 3):
        raise RuntimeError(f"oracle check_image: invalid input (status {rc})")
    return rc == 0, msg.value.decode(), _counts_dict(c)


def check_chain_image(schema, src_root: int, image: np.ndarray, dev_base: int, path, x_field: int,
                      y_field: int = -1, root_off: int = 0):
    """Check a host copy of a device arena that holds a selective deep copy of
    one chain (the struct blocks it passes through, the x / y arrays of the
    struct it reaches) against the source tree, along that chain only."""
    image = np.ascontiguousarray(image, dtype=np.uint8)
    steps = _steps(path)
    msg = ctypes.create_string_buffer(1024)
    rc = lib().or_check_chain_image(ctypes.byref(_cs(schema).struct), src_root, image.ctypes.data, image.nbytes,
                                    dev_base, root_off, steps, len(path), x_field, y_field, msg, 1024)
    if rc not in (0, 3):
        raise RuntimeError(f"oracle check_chain_image: invalid input (status {rc})")
    return rc == 0, msg.value.decode()


def image_resolve(schema, image: np.ndarray, dev_base: int, path, root_off: int = 0) -> int:
    image = np.ascontiguousarray(image, dtype=np.uint8)
    steps = _steps(path)
    out = ctypes.c_uint64()
    _check(lib().or_image_resolve(ctypes.byref(_cs(schema).struct), image.ctypes.data, image.nbytes,
                                  dev_base, root_off, steps, len(path), ctypes.byref(out)),
           "image_resolve")
    return out.value


def host_resolve(schema, root: int, path) -> int:
    steps = _steps(path)
    out = ctypes.c_uint64()
    _check(lib().or_host_resolve(ctypes.byref(_cs(schema).struct), root, steps, len(path),
                                 ctypes.byref(out)), "host_resolve")
    return out.value
