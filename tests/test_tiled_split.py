"""The temporal-blocking kernel's split of a grid into (chunk, strip) work
items, computed by the library's host code (flood_debug_tiled_split; no GPU).

Large grids get about eight items per pipeline of at least 24 K rows, handed
out by a launch counter; grids too small for four such items per pipeline get
the round-robin split whose chunk count minimises the busiest pipeline's
ticks, (items per pipeline) x (rows + 3K - 1).  The split is memoised per
thread, so handles stepped from several threads cannot see each other's.
"""
import math
import threading

import pytest


def F():
    import paper_2204_10323_gb300 as F
    return F


# output columns of a 128-column strip: less a 4-column halo on each side for
# K <= 4, 8 for K = 8; the theta weighting reaches K + 1 columns to the right,
# rounded up to 4 (so it widens the right halo for K = 4 and 8 only)
STRIP = {(4, 0): 120, (4, 1): 116, (4, 2): 120, (4, 3): 116, (8, 0): 112, (8, 1): 108, (1, 0): 120, (2, 3): 120}


def strip_width(K, mode):
    return STRIP[(K, mode)]


@pytest.mark.parametrize("K,mode", [(4, 0), (4, 1), (4, 2), (8, 0), (1, 0), (2, 3)])
def test_items_cover_the_grid(K, mode):
    Fm = F()
    for nx, ny in [(1, 1), (7, 5), (300, 40), (1024, 1024), (2048, 2048), (1100, 2300), (4096, 4096),
                   (8192, 8192), (16384, 16384), (3, 600000)]:
        r = Fm.flood_debug_tiled_split(nx, ny, K, mode, 912)
        assert r["chunk_rows"] >= 1
        strips = math.ceil(nx / strip_width(K, mode))
        assert r["items"] == strips * math.ceil(ny / r["chunk_rows"]), (nx, ny)
        assert r["blocks"] == min(r["items"], 912)


def test_large_grids_get_eight_items_per_pipeline():
    Fm = F()
    assert Fm.flood_debug_tiled_split(16384, 16384)["chunk_rows"] == 304     # the measured best at 16384^2
    assert Fm.flood_debug_tiled_split(8192, 8192)["chunk_rows"] == 96
    for n in (8192, 12000, 16384, 30000):
        r = Fm.flood_debug_tiled_split(n, n)
        assert r["chunk_rows"] >= 24 * 4
        assert 4 * 912 <= r["items"] <= 9 * 912 + math.ceil(n / 120), n


def test_small_grids_minimise_the_busiest_pipelines_ticks():
    Fm = F()
    K, resident = 4, 912
    for nx, ny in [(1024, 1024), (2048, 2048), (4096, 4096), (300, 40), (2000, 700)]:
        r = Fm.flood_debug_tiled_split(nx, ny, K, 0, resident)
        strips = math.ceil(nx / 120)

        def ticks(rows):
            items = strips * math.ceil(ny / rows)
            return math.ceil(items / resident) * (rows + 3 * K - 1)
        candidates = {math.ceil(ny / c) for c in range(1, (ny + 15) // 16 + 1)}
        assert ticks(r["chunk_rows"]) == min(ticks(rows) for rows in candidates), (nx, ny)


def test_split_is_the_same_from_many_threads():
    Fm = F()
    cases = [(nx, ny, K) for nx, ny in [(1024, 1024), (300, 40), (2048, 2048), (777, 333), (4096, 512)]
             for K in (1, 2, 4)]
    want = {c: Fm.flood_debug_tiled_split(c[0], c[1], c[2]) for c in cases}
    bad = []

    def worker(offset):
        for it in range(300):
            c = cases[(offset + it) % len(cases)]
            if Fm.flood_debug_tiled_split(c[0], c[1], c[2]) != want[c]:
                bad.append(c)
    threads = [threading.Thread(target=worker, args=(k,)) for k in range(8)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not bad


@pytest.mark.parametrize("args", [(0, 5, 4, 0, 912), (5, 0, 4, 0, 912), (5, 5, 5, 0, 912), (5, 5, 4, 4, 912),
                                  (5, 5, 4, 0, 0)])
def test_bad_arguments(args):
    Fm = F()
    with pytest.raises(Fm.FloodError):
        Fm.flood_debug_tiled_split(*args)
