"""The grouping key of the adjoint's warp reduce-scatter, written out on the
host exactly as trace_bwd_kernel forms it, over every cell of every level
and volume that has a valid corner: no two cells may share a key (lanes with
one key are summed onto the corners of one cell).  Cells inside a level are
keyed by their Morton code plus the level's and the volume's texel offsets;
cells whose lower corner lies at -1 on some axes by bit 31, that axis mask
and the offset code of the cell moved to 0 on them."""
import itertools

import pytest

M = 0x09249249  # Morton bits of x: 0, 3, ..., 27 (10 coordinate bits)


def spread(v):
    r = 0
    for b in range(10):
        r |= ((v >> b) & 1) << (3 * b)
    return r


def spread_inc(s, m):
    return (s - m) & m  # spread(v + 1) from spread(v), 10-bit wrap


def all_keys(n, aniso):
    levels = n.bit_length()
    off, acc = [], 0
    for l in range(levels):
        off.append(acc)
        acc += (n >> l) ** 3 * (6 if aniso and l >= 1 else 1)
    keys = {}
    for l in range(levels):
        nl = n >> l
        for vol in range(6 if aniso and l >= 1 else 1):
            vbase = vol * nl ** 3
            for b in itertools.product(range(-1, nl), repeat=3):
                ok = [[0 <= b[a] + d < nl for d in (0, 1)] for a in range(3)]
                valid = sum(1 << c for c in range(8)
                            if ok[0][c & 1] and ok[1][(c >> 1) & 1] and ok[2][c >> 2])
                if valid == 0:
                    continue  # nothing to scatter: the kernel leaves the lane out
                sx0, sy0, sz0 = spread(b[0] & 1023), spread(b[1] & 1023) << 1, spread(b[2] & 1023) << 2
                if valid & 1:
                    key = off[l] + vbase + (sx0 | sy0 | sz0)
                else:
                    assert acc < 0x0fffff00
                    mx = 1 if sx0 == M else 0
                    my = 2 if sy0 == M << 1 else 0
                    mz = 4 if sz0 == M << 2 else 0
                    cell = ((spread_inc(sx0, M) if mx else sx0) | (spread_inc(sy0, M << 1) if my else sy0)
                            | (spread_inc(sz0, M << 2) if mz else sz0))
                    key = 0x80000000 | ((mx | my | mz) << 28) | (off[l] + vbase + cell)
                assert 0 <= key < 0xffffff00, key  # below the per-lane and inactive keys
                assert key not in keys, (key, (l, vol, b), keys[key])
                keys[key] = (l, vol, b)
    return keys


@pytest.mark.parametrize("n,aniso", [(2, False), (8, False), (16, False), (2, True), (8, True),
                                     (16, True)])
def test_keys_unique(n, aniso):
    keys = all_keys(n, aniso)
    assert len(keys) > n ** 3


def test_packed_keys_fit_up_to_512():
    """The packed keys need every offset below 0x0fffff00 (then the largest,
    mask 7, stays below the per-lane keys 0xffffff00 + lane): true for
    n <= 512 in both layouts; the kernel falls back to per-lane keys beyond,
    and the in-range keys of n = 1024 stay below 2^31."""
    for aniso in (False, True):
        total = sum((512 >> l) ** 3 * (6 if aniso and l >= 1 else 1) for l in range(10))
        assert total < 0x0fffff00
        assert (0x80000000 | (7 << 28) | (total - 1)) < 0xffffff00
        big = sum((1024 >> l) ** 3 * (6 if aniso and l >= 1 else 1) for l in range(11))
        assert 0x0fffff00 <= big < 1 << 31
