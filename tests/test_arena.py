"""Host logic of the serving arena: the first-fit free list never hands out
overlapping or unaligned chunks, never exceeds its size, coalesces freed
neighbours, and refuses what cannot be placed.  Checked against a byte map
on random alloc/free sequences (CPU only)."""
import numpy as np

from paper_2403_20190_gb300.arena import ALIGN, FreeList


def test_random_sequences_against_a_byte_map():
    rng = np.random.default_rng(5)
    for trial in range(20):
        size = int(rng.integers(1, 64)) * ALIGN * 16 + int(rng.integers(0, ALIGN))
        fl = FreeList(size)
        assert fl.size % ALIGN == 0 and fl.size <= size
        owner = np.full(fl.size, -1, dtype=np.int64)
        live = {}
        for step in range(300):
            if live and rng.random() < 0.45:
                off = list(live)[int(rng.integers(len(live)))]
                fl.free(off)
                owner[off:off + live.pop(off)] = -1
            else:
                want = int(rng.integers(1, fl.size // 3 + 2))
                off = fl.alloc(want)
                n = -(-want // ALIGN) * ALIGN
                # a fit exists iff some aligned free run of n bytes exists
                free = owner == -1
                fits = any(free[o:o + n].all() and o + n <= fl.size for o in range(0, fl.size, ALIGN))
                if off is None:
                    assert not fits
                    continue
                assert off % ALIGN == 0 and off + n <= fl.size
                assert (owner[off:off + n] == -1).all(), "overlap"
                owner[off:off + n] = step
                live[off] = n
            assert fl.free_bytes == int((owner == -1).sum())
        for off in list(live):
            fl.free(off)
        assert fl.free_bytes == fl.size and fl.largest_free == fl.size


def test_budget_is_a_cap():
    fl = FreeList(10 * ALIGN + 7)
    assert fl.size == 10 * ALIGN
    assert fl.alloc(10 * ALIGN + 1) is None
    a = fl.alloc(4 * ALIGN)
    b = fl.alloc(6 * ALIGN)
    assert (a, b) == (0, 4 * ALIGN) and fl.alloc(1) is None
    fl.free(a)
    assert fl.alloc(5 * ALIGN) is None and fl.alloc(4 * ALIGN) == 0
