"""CPU tests of the serving loop's admission allocator (no GPU calls)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def drr():
    from paper_2208_12737_gb300 import build
    build.build()
    from paper_2208_12737_gb300 import drr as d
    d.load()
    return d


def test_first_fit_alignment_and_exhaustion(drr):
    a = drr.Arena(4096, 256)
    offs = [a.alloc(100) for _ in range(16)]
    assert offs == [256 * i for i in range(16)]
    assert a.in_use() == 4096 and a.largest_free() == 0
    with pytest.raises(drr.DrrError) as ei:
        a.alloc(1)
    assert ei.value.status == 2  # DRR_ERR_OOM
    a.close()


def test_coalescing_and_reuse(drr):
    a = drr.Arena(1 << 20, 256)
    blocks = [a.alloc(1000) for _ in range(100)]
    for off in blocks[::2]:
        a.free(off)
    assert a.largest_free() >= (1 << 20) - 100 * 1024  # the tail run
    for off in blocks[1::2]:
        a.free(off)
    assert a.in_use() == 0 and a.largest_free() == 1 << 20  # everything merged back
    with pytest.raises(drr.DrrError) as ei:
        a.free(12345)
    assert ei.value.status == 6  # DRR_ERR_NOT_FOUND
    a.close()


def test_random_alloc_free_matches_model(drr):
    rng = np.random.default_rng(0)
    cap = 1 << 16
    a = drr.Arena(cap, 64)
    live = {}
    for _ in range(2000):
        if live and rng.uniform() < 0.45:
            off = list(live)[rng.integers(len(live))]
            a.free(off)
            del live[off]
        else:
            n = int(rng.integers(1, 3000))
            try:
                off = a.alloc(n)
            except drr.DrrError:
                continue
            size = (n + 63) // 64 * 64
            assert off % 64 == 0 and off + size <= cap
            for o, s in live.items():  # no overlap with any live block
                assert off + size <= o or o + s <= off
            live[off] = size
        assert a.in_use() == sum(live.values())
    a.close()
