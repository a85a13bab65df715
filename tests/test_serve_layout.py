"""Host-side invariants of the serving tick table (no GPU): the layout the
server builds for a tick gives each admitted request a contiguous, ascending
range of warp tiles and of poses, and together the ranges cover the tick
exactly once, so the kernels' decode of any tile or pose index (binary search
over the starts, then pose = local index // tiles per pose) always lands
inside the request that owns it."""
import ctypes

import numpy as np
import pytest

from paper_2208_12737_gb300 import build


@pytest.fixture(scope="module")
def lib():
    build.build()
    from paper_2208_12737_gb300 import drr
    return drr.load()


def _tiles_per_pose(H, W):
    return -(-W // 8) * -(-H // 4)


def _layout(lib, Bs, dets):
    from paper_2208_12737_gb300 import drr
    n = len(Bs)
    B = (ctypes.c_int32 * n)(*Bs)
    D = (drr.drr_detector * n)(*[drr.detector(d) for d in dets])
    ts, ps, tot = (ctypes.c_int32 * n)(), (ctypes.c_int32 * n)(), (ctypes.c_int32 * 2)()
    st = lib.drr_serve_tick_layout(n, B, D, ts, ps, tot)
    return st, np.array(ts), np.array(ps), tuple(tot)


def _find(starts, i):
    """The kernels' decode: the last request whose start is <= i."""
    lo, hi = 0, len(starts) - 1
    while lo < hi:
        mid = (lo + hi + 1) >> 1
        if starts[mid] <= i:
            lo = mid
        else:
            hi = mid - 1
    return lo


@pytest.mark.parametrize("seed", range(6))
def test_tick_layout_covers_every_tile_and_pose_once(lib, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 40))
    Bs = [int(b) for b in rng.integers(1, 6, n)]
    dets = [(510.0, int(h), int(w), 1.0, 1.0) for h, w in rng.integers(1, 90, (n, 2))]
    st, ts, ps, (tt, tp) = _layout(lib, Bs, dets)
    assert st == 0
    per = [_tiles_per_pose(d[1], d[2]) for d in dets]
    assert tt == sum(b * p for b, p in zip(Bs, per)) and tp == sum(Bs)
    assert ts[0] == 0 and ps[0] == 0
    assert np.all(np.diff(ts) > 0) and np.all(np.diff(ps) > 0)
    owner = np.full(tt, -1)
    for i in range(n):
        owner[ts[i]:ts[i] + Bs[i] * per[i]] = i
    assert np.all(owner >= 0)  # contiguous ranges, no gap, no overlap
    for t in range(tt):  # every tile decodes to a pose of the request that owns it
        r = _find(ts, t)
        assert r == owner[t]
        assert 0 <= (t - ts[r]) // per[r] < Bs[r]
    for p in range(tp):
        r = _find(ps, p)
        assert 0 <= p - ps[r] < Bs[r]


def test_tick_layout_rejects_bad_requests(lib):
    assert _layout(lib, [0], [(510.0, 8, 8, 1.0, 1.0)])[0] == 1
    assert _layout(lib, [1], [(510.0, 0, 8, 1.0, 1.0)])[0] == 1
    # a layout past 2^31 tiles is refused instead of wrapping
    assert _layout(lib, [65535] * 2, [(510.0, 32768, 32768, 1.0, 1.0)] * 2)[0] == 1
