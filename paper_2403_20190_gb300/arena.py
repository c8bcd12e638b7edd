"""A device arena for the serving loop: one allocation made up front, carved
into per-batch chunks by a first-fit free list with coalescing.

The request loop admits a batch only when its whole footprint (encrypted
samples, scratch, responses) can be placed in the arena, so the HBM budget is
enforced physically and nothing in the loop calls the CUDA allocator.  A
chunk is returned only after the batch's completion event has fired, so it
can be reused by any stream without further ordering.
"""
import bisect

import torch

ALIGN = 256


def align_up(x: int, a: int = ALIGN) -> int:
    return (int(x) + a - 1) // a * a


class FreeList:
    """First-fit allocator over [0, size) bytes; blocks are ALIGN-aligned.
    Pure host bookkeeping."""

    def __init__(self, size: int):
        self.size = int(size) // ALIGN * ALIGN  # the budget is a cap: round down
        self._off = [0]            # free blocks, sorted by offset
        self._len = [self.size]
        self.used = {}             # offset -> length of live chunks

    @property
    def free_bytes(self) -> int:
        return sum(self._len)

    @property
    def largest_free(self) -> int:
        return max(self._len, default=0)

    def alloc(self, nbytes: int):
        """Offset of a chunk of at least nbytes, or None if no free block fits."""
        n = align_up(max(int(nbytes), 1))
        for k, ln in enumerate(self._len):
            if ln >= n:
                off = self._off[k]
                if ln == n:
                    del self._off[k]
                    del self._len[k]
                else:
                    self._off[k] += n
                    self._len[k] -= n
                self.used[off] = n
                return off
        return None

    def free(self, off: int):
        n = self.used.pop(off)
        k = bisect.bisect_left(self._off, off)
        self._off.insert(k, off)
        self._len.insert(k, n)
        # merge with the right neighbour, then the left
        if k + 1 < len(self._off) and self._off[k] + self._len[k] == self._off[k + 1]:
            self._len[k] += self._len.pop(k + 1)
            self._off.pop(k + 1)
        if k > 0 and self._off[k - 1] + self._len[k - 1] == self._off[k]:
            self._len[k - 1] += self._len.pop(k)
            self._off.pop(k)


class DeviceArena:
    """FreeList over one uint8 device tensor; chunks come back as a Chunk that
    hands out typed, aligned sub-buffers."""

    def __init__(self, nbytes: int, device):
        self.fl = FreeList(nbytes)
        self.buf = torch.empty(self.fl.size, dtype=torch.uint8, device=device)

    @property
    def size(self):
        return self.fl.size

    @property
    def free_bytes(self):
        return self.fl.free_bytes

    def alloc(self, nbytes: int):
        off = self.fl.alloc(nbytes)
        return None if off is None else Chunk(self, off, align_up(max(int(nbytes), 1)))

    def release(self, chunk):
        self.fl.free(chunk.off)


class Chunk:
    def __init__(self, arena, off, nbytes):
        self.arena, self.off, self.nbytes, self.cur = arena, off, nbytes, 0

    def take(self, count: int, dtype: torch.dtype):
        """The next ALIGN-aligned sub-buffer of `count` elements."""
        esz = torch.empty((), dtype=dtype).element_size()
        nb = align_up(int(count) * esz)
        if self.cur + nb > self.nbytes:
            raise ValueError("chunk overflow: layout and footprint disagree")
        s = self.off + self.cur
        self.cur += nb
        return self.arena.buf[s:s + int(count) * esz].view(dtype)
