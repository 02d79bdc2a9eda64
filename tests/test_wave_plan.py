"""CPU checks of the wavefront sweeps' unit tables (sn_wave_plan, host code of the
library, no GPU call).  The sweep of Sec. 2 solves a cell after its three upwind
neighbours; the wavefront kernels hand out tiles of (cell, group) keys in order and
let each tile wait only for the units its two dependency ranges name.  A range that
missed an upwind tile would be a race (a cell read before its neighbour wrote its
face), so the ranges are checked here by brute force against hyperplanes rebuilt
from their definition, over odd mesh shapes, group counts and SM counts."""
import ctypes

import numpy as np
import pytest

KEY_BLOCK = 128      # threads of a wavefront CTA: keys of a tile x chunks a key
MIN_BLOCKS = 3       # resident CTAs an SM the chunk rule counts


@pytest.fixture(scope="module")
def sn():
    from paper_1906_04017_gb300 import build, sn as mod
    build.build()
    return mod


def hyperplanes(nx, ny, nz):
    """Cells (i, j, k) of each hyperplane i+j+k = s, listed by (k, j, i)."""
    planes = [[] for _ in range(nx + ny + nz - 2)]
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                planes[i + j + k].append((i, j, k))
    return planes


def chunks_log2(keys, Do, nsm):
    """The fewest chunks (a power of two, at most 8 and at most Do) for which
    keys x chunks fills the GPU's resident thread slots, else the most allowed."""
    most = min(3, Do.bit_length() - 1)
    for l in range(most + 1):
        if keys * (1 << l) >= nsm * MIN_BLOCKS * KEY_BLOCK:
            return l
    return most


def check_plan(sn, nx, ny, nz, G, Do, nsm):
    units, uplane = sn.wave_plan(nx, ny, nz, G, Do, nsm)
    planes = hyperplanes(nx, ny, nz)
    place = {c: q for pl in planes for q, c in enumerate(pl)}
    first = {}                       # (s, octant) -> first unit, tile size, tiles
    u = 0
    off = 0
    for s, pl in enumerate(planes):
        n = len(pl)
        lch = chunks_log2(8 * n * G, Do, nsm)
        kb = KEY_BLOCK >> lch
        ntile = -(-n * G // kb)
        for o in range(8):
            first[s, o] = (u, kb, ntile)
            for tl in range(ntile):
                assert units[u, 0] == tl * kb, (s, o, tl)
                assert units[u, 1] == s | (o << 12) | (lch << 15), (s, o, tl)
                assert list(uplane[u, :2]) == [off, n * G], (s, o, tl)
                u += 1
        off += n
    assert u == len(units) == len(uplane)

    for s in range(1, len(planes)):
        pl = planes[s]
        n = len(pl)
        _, kb, ntile = first[s, 0]
        kbp = first[s - 1, 0][1]
        for tl in range(ntile):
            need, near = set(), set()   # tiles holding an upwind key; any key of an upwind cell
            for key in range(tl * kb, min(tl * kb + kb, n * G)):
                i, j, k = pl[key // G]
                g = key % G
                for nb in ((i - 1, j, k), (i, j - 1, k), (i, j, k - 1)):
                    if min(nb) < 0:
                        continue
                    p = place[nb]
                    assert sum(nb) == s - 1
                    need.add((p * G + g) // kbp)
                    near.update(range(p * G // kbp, (p * G + G - 1) // kbp + 1))
            assert need, (s, tl)
            for o in range(8):
                u = first[s, o][0] + tl
                base, _, ntp = first[s - 1, o]
                lo1, n1 = int(units[u, 2]), int(units[u, 3])
                lo2, n2 = int(uplane[u, 2]), int(uplane[u, 3])
                assert n1 >= 1 and n2 >= 0
                covered = set(range(lo1, lo1 + n1)) | set(range(lo2, lo2 + n2))
                # every upwind tile of the same octant is waited for ...
                missing = {base + t for t in need} - covered
                assert not missing, (s, o, tl, sorted(missing))
                # ... the ranges stay in hyperplane s - 1 of the same octant (so every
                # wait is on a unit handed out earlier) ...
                for lo, cnt in ((lo1, n1), (lo2, n2)):
                    if cnt:
                        assert base <= lo and lo + cnt <= base + ntp, (s, o, tl)
                # ... and each range starts and ends on a tile of an upwind cell
                for lo, cnt in ((lo1, n1), (lo2, n2)):
                    if cnt:
                        assert lo - base in near and lo + cnt - 1 - base in near, (s, o, tl)
                if n2:
                    assert lo2 > lo1 + n1, (s, o, tl)
    for o in range(8):
        u0, _, nt0 = first[0, o]
        assert not units[u0:u0 + nt0, 3].any() and not uplane[u0:u0 + nt0, 3].any()


@pytest.mark.parametrize("nx,ny,nz,G,Do,nsm", [
    (1, 1, 1, 1, 1, 1),
    (5, 7, 3, 2, 10, 4),
    (12, 10, 11, 3, 3, 152),
    (3, 1, 9, 8, 36, 1),
    (1, 1, 40, 5, 6, 2),
    (33, 2, 5, 1, 21, 16),
    (16, 16, 16, 8, 10, 152),
    (9, 13, 6, 17, 15, 7),
    (8, 8, 8, 64, 64, 1000),
    (24, 24, 24, 2, 10, 152),
])
def test_wave_plan_covers_every_upwind_dependency(sn, nx, ny, nz, G, Do, nsm):
    check_plan(sn, nx, ny, nz, G, Do, nsm)


def test_wave_plan_chunks_follow_the_gpu_size(sn):
    """On the same mesh, a GPU with more SMs gets more chunks a key on the same
    hyperplane (smaller tiles, more units), never fewer."""
    small, _ = sn.wave_plan(12, 12, 12, 4, 10, 8)
    big, _ = sn.wave_plan(12, 12, 12, 4, 10, 152)
    assert len(big) >= len(small) > 0
    lch_small = {(int(r[1]) & 4095): int(r[1]) >> 15 for r in small}
    lch_big = {(int(r[1]) & 4095): int(r[1]) >> 15 for r in big}
    assert all(lch_big[s] >= lch_small[s] for s in lch_small)
    assert max(lch_big.values()) == 3 and min(lch_small.values()) < 3


@pytest.mark.parametrize("args", [
    (0, 4, 4, 1, 10, 152), (1024, 4, 4, 1, 10, 152), (4, 4, 4, 0, 10, 152),
    (4, 4, 4, 1025, 10, 152), (4, 4, 4, 1, 0, 152), (4, 4, 4, 1, 65, 152), (4, 4, 4, 1, 10, 0),
])
def test_wave_plan_rejects_bad_sizes(sn, args):
    n = ctypes.c_int64(-1)
    assert sn.lib().sn_wave_plan(*args, None, None, 0, ctypes.byref(n)) == sn.SN_EINVAL
    assert n.value == 0
    assert sn.lib().sn_last_error(None)


def test_wave_plan_rejects_a_short_output(sn):
    n = ctypes.c_int64()
    assert sn.lib().sn_wave_plan(4, 4, 4, 2, 10, 152, None, None, 0, ctypes.byref(n)) == sn.SN_OK
    assert n.value > 1
    buf = np.zeros((n.value, 4), dtype=np.int32)
    p = buf.ctypes.data_as(ctypes.c_void_p)
    assert sn.lib().sn_wave_plan(4, 4, 4, 2, 10, 152, p, p, n.value - 1, ctypes.byref(n)) == sn.SN_EINVAL
    assert sn.lib().sn_wave_plan(4, 4, 4, 2, 10, 152, p, None, n.value, ctypes.byref(n)) == sn.SN_EINVAL
