"""Pure-Python readers for host memory, used by tests to inspect trees without
going through either the oracle or the CUDA path."""
from __future__ import annotations

import ctypes
import struct

import numpy as np


def read(addr: int, nbytes: int) -> bytes:
    return ctypes.string_at(addr, nbytes)


def u64(addr: int) -> int:
    return struct.unpack("<Q", read(addr, 8))[0]


def i32(addr: int) -> int:
    return struct.unpack("<i", read(addr, 4))[0]


def f32_view(addr: int, n: int) -> np.ndarray:
    if n == 0:
        return np.zeros(0, dtype=np.float32)
    return np.ctypeslib.as_array((ctypes.c_float * n).from_address(addr))


def f64_view(addr: int, n: int) -> np.ndarray:
    if n == 0:
        return np.zeros(0, dtype=np.float64)
    return np.ctypeslib.as_array((ctypes.c_double * n).from_address(addr))


def node_walk(root: int):
    """Preorder walk of a node-struct tree ``{int32 n; int32 nchild; float*
    position; float* velocity; Node* child}``.  Yields dicts with the node's
    path (tuple of child indices), address, scalars and pointers."""
    stack = [((), root)]
    while stack:
        path, a = stack.pop()
        n, nchild = i32(a), i32(a + 4)
        node = dict(path=path, addr=a, n=n, nchild=nchild, pos=u64(a + 8), vel=u64(a + 16),
                    child=u64(a + 24), raw=read(a, 32))
        yield node
        for j in reversed(range(nchild)):
            stack.append((path + (j,), node["child"] + 32 * j))


def node_arrays(root: int):
    """{path: (position copy, velocity copy)} for every node of a node tree."""
    out = {}
    for nd in node_walk(root):
        out[nd["path"]] = (f32_view(nd["pos"], nd["n"]).copy(), f32_view(nd["vel"], nd["n"]).copy())
    return out


def half_axpy_exact(p: np.ndarray, v: np.ndarray) -> np.ndarray:
    """p + 0.5*v rounded once to fp32: for fp32 inputs the exact sum has at
    most 26 significant bits, so fp64 holds it exactly and the single cast to
    fp32 is the correctly rounded IEEE-754 result."""
    return (p.astype(np.float64) + 0.5 * v.astype(np.float64)).astype(np.float32)


def same_bits(a: np.ndarray, b: np.ndarray) -> bool:
    return a.shape == b.shape and a.tobytes() == b.tobytes()
