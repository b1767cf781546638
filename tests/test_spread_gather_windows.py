"""CPU mirror of the spread's gather walk (ibdl_device.cuh, phase_rows_fwd
stage B): for sorted tile bins, every (point, node) pair of a point's 6 x 6
support box that falls in the tile is visited exactly once, by the lane that
owns the node, whatever the grid size, tiling, warp count, chunk size and
periodic wrap.  The GPU parity tests pin the kernel's values; this pins its
index arithmetic (column groups, candidate windows, the wrapped run near
x = n, and the skip to the next group that can have a candidate).
"""
import numpy as np
import pytest

BOX = 6


def lower_bound(sx, p, v):
    while p < len(sx) and sx[p] < v:
        p += 1
    return p


def gather_visits(n, R, xs, yb, y0, nwarps):
    """Mirror of stage B for one chunk: returns {(point, row, col): count}."""
    np_ = len(xs)
    lgR = R.bit_length() - 1
    cpg = 32 >> lgR
    ncg = n // cpg
    mask = n - 1
    visits = {}
    allwin = cpg + BOX - 1 >= n
    for warp in range(nwarps):
        plo = phi = 0
        gi = warp
        while gi < ncg:
            x0 = gi * cpg
            w0 = w1 = np_
            if allwin:
                e0, e1 = 0, np_
            else:
                wl = x0 - (BOX - 1)
                plo = lower_bound(xs, plo, 0 if wl < 0 else wl)
                phi = lower_bound(xs, phi if phi > plo else plo, x0 + cpg)
                e0, e1 = plo, phi
                if wl < 0:
                    w0 = lower_bound(xs, phi, n + wl)
                if e0 == e1 and w0 == w1:
                    if plo >= np_:
                        break
                    first = xs[plo]
                    gneed = int((first - cpg + 1) / cpg)  # C++ truncation toward zero
                    if gneed > gi + nwarps:
                        gi += ((gneed - gi) // nwarps) * nwarps - nwarps
                    gi += nwarps
                    continue
            for lane in range(32):
                lr, lc = lane & (R - 1), lane >> lgR
                x = x0 + lc
                yrow = y0 + lr
                for ea, eb in ((e0, e1), (w0, w1)):
                    for e in range(ea, eb):
                        a = (x - xs[e]) & mask
                        bb = (yrow - yb[e]) & mask
                        if a < BOX and bb < BOX:
                            key = (e, lr, x)
                            visits[key] = visits.get(key, 0) + 1
            gi += nwarps
    return visits


def expected_pairs(n, R, xs, yb, y0):
    out = set()
    for e, (x, y) in enumerate(zip(xs, yb)):
        for a in range(BOX):
            for bb in range(BOX):
                r = (y + bb - y0) % n
                if r < R:
                    out.add((e, r, (x + a) % n))
    return out


@pytest.mark.parametrize("n,R", [(16, 2), (16, 4), (16, 8), (32, 4), (64, 8), (64, 16),
                                 (128, 32), (256, 4), (1024, 4), (2048, 2)])
@pytest.mark.parametrize("layout", ["random", "cluster_left", "cluster_right", "wrap", "dense"])
def test_every_box_node_is_visited_once(n, R, layout):
    rng = np.random.default_rng(n * 100 + R)
    y0 = int(rng.integers(0, n // R)) * R
    k = 60
    if layout == "random":
        xs = rng.integers(0, n, k)
    elif layout == "cluster_left":
        xs = rng.integers(0, min(n, 8), k)
    elif layout == "cluster_right":
        xs = rng.integers(max(0, n - 8), n, k)
    elif layout == "wrap":
        xs = np.concatenate([rng.integers(0, 3, k // 2), rng.integers(n - 3, n, k // 2)])
    else:
        xs = rng.integers(n // 2 - 2, n // 2 + 2, k)
    # rows within reach of the tile (the bin's rule), some across the wrap
    yb = (y0 + rng.integers(-(BOX - 1), R, len(xs))) % n
    order = np.lexsort((np.arange(len(xs)), xs))
    xs, yb = [int(v) for v in xs[order]], [int(v) for v in yb[order]]
    for nwarps in (1, 3, 8):
        got = gather_visits(n, R, xs, yb, y0, nwarps)
        assert all(c == 1 for c in got.values()), "a node visited twice"
        assert set(got) == expected_pairs(n, R, xs, yb, y0), (n, R, layout, nwarps)
