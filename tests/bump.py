"""A bump allocator for treegen trees in tests: every block from one ctypes buffer, 16-byte
aligned, `gap` bytes after the block before it, so that a tree's host layout is known (and
compact, whatever the process heap looks like)."""
import ctypes

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64)


class BumpAllocator:
    """`min_align` of 8 places every block on 8 bytes instead of the 16 that treegen asks for, as
    a packing allocator would (enough for the node trees' pointers, ints, floats and doubles), so
    that blocks lie at host addresses off 16-byte boundaries."""

    def __init__(self, nbytes, gap=0, min_align=16):
        self.buf = (ctypes.c_uint8 * (nbytes + 64))()
        self.next = (ctypes.addressof(self.buf) + 15) // 16 * 16 + (16 - min_align) % 16
        self.end = ctypes.addressof(self.buf) + nbytes
        self.gap, self.blocks, self.min_align = gap, [], min_align
        self.fn = ALLOC_FN(self._alloc)

    def _alloc(self, ctx, nbytes, align):
        al = self.min_align if self.min_align < 16 else max(align, 16)
        a = (self.next + al - 1) // al * al
        if a + nbytes > self.end:
            return None
        self.next = a + nbytes + self.gap
        if nbytes:
            self.blocks.append((a, nbytes))
        return a

    @property
    def alloc(self):
        """The (function address, context) pair treegen takes."""
        return (ctypes.cast(self.fn, ctypes.c_void_p).value, None)
