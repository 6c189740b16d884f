"""Pipeline model and chunk-schedule search of the host-buffer path.

Host logic only (no GPU): makespans worked by hand for small schedules, the
wave factor of the persistent kernel, and the searched schedule against
lower bounds that hold for every schedule.
"""

import itertools
import math

import pytest

import paper_2203_14906_gb300 as pa


def model(**kw):
    base = dict(items_per_frame=1, resident=1, upload_us=1.0, kernel_us=2.0, download_us=3.0,
                launch_us=0.5, wave_share=1.0, n_sets=3)
    base.update(kw)
    return base


def test_two_chunks_by_hand():
    # chunk 0: up 0-1, launch sequence 1-3.5, down 3.5-6.5
    # chunk 1: up 1-2, launch sequence 3.5-6 (after chunk 0's), down 6.5-9.5
    assert pa.pipe_time([1, 1], **model()) == pytest.approx(9.5, abs=1e-12)
    # one buffer set: chunk 1's upload waits for chunk 0's download (6.5)
    # up 6.5-7.5, launch sequence 7.5-10, down 10-13
    assert pa.pipe_time([1, 1], **model(n_sets=1)) == pytest.approx(13.0, abs=1e-12)
    # three frames in one chunk: 3 + 6 + 0.5 + 9
    assert pa.pipe_time([3], **model()) == pytest.approx(18.5, abs=1e-12)
    assert pa.pipe_time([], **model()) == 0.0


def test_wave_factor():
    # 3 frames x 256 items on 608 resident blocks: 1.263 waves run as 2
    w = 3 * 256 / 608
    m = model(items_per_frame=256, resident=608, upload_us=0.0, download_us=0.0, launch_us=0.0,
              kernel_us=10.0)
    assert pa.pipe_time([3], **m) == pytest.approx(2 * 10.0 * 608 / 256, rel=1e-12)
    m["wave_share"] = 0.5
    assert pa.pipe_time([3], **m) == pytest.approx(30.0 * (0.5 + 0.5 * 2 / w), rel=1e-12)
    m["wave_share"] = 0.0
    assert pa.pipe_time([3], **m) == pytest.approx(30.0, rel=1e-12)
    # 19 frames fill exactly 8 waves: no loss at any wave share
    m["wave_share"] = 1.0
    assert pa.pipe_time([19], **m) == pytest.approx(190.0, rel=1e-12)


def _valid(s, n, cap):
    assert sum(s) == n and all(1 <= c <= cap for c in s), s


@pytest.mark.parametrize("n,cap", [(1, 1), (5, 2), (32, 32), (64, 64), (100, 16)])
def test_copy_bound_schedule_reaches_the_lower_bound(n, cap):
    """Free kernels: every schedule needs the first frame's upload and all
    downloads one after another, th + n td; one-frame chunks reach it."""
    m = model(kernel_us=0.0, launch_us=0.0, upload_us=1.0, download_us=3.0)
    s = pa.pipe_schedule(n, cap, **m)
    _valid(s, n, cap)
    assert pa.pipe_time(s, **m) == pytest.approx(1.0 + 3.0 * n, rel=1e-12)


@pytest.mark.parametrize("n,cap", [(6, 8), (20, 32), (40, 16)])
def test_free_copies_favour_few_chunks(n, cap):
    """Free copies and a per-chunk launch cost: fewest chunks win."""
    m = model(upload_us=0.0, download_us=0.0, kernel_us=2.0, launch_us=5.0, wave_share=0.0)
    s = pa.pipe_schedule(n, cap, **m)
    _valid(s, n, cap)
    assert len(s) == math.ceil(n / cap)
    assert pa.pipe_time(s, **m) == pytest.approx(2.0 * n + 5.0 * len(s), rel=1e-12)


def _compositions(n, cap):
    for k in range(1, n + 1):
        for cut in itertools.combinations(range(1, n), k - 1):
            parts = [b - a for a, b in zip((0,) + cut, cut + (n,))]
            if max(parts) <= cap:
                yield parts


@pytest.mark.parametrize("ratio", [0.5, 1.0, 1.6, 3.0])
def test_search_close_to_exhaustive_optimum(ratio):
    """12 frames: the searched family's best against every composition."""
    m = model(items_per_frame=256, resident=608, upload_us=4.9, download_us=16.4,
              kernel_us=16.4 * ratio, launch_us=20.0, wave_share=0.5)
    s = pa.pipe_schedule(12, 12, **m)
    _valid(s, 12, 12)
    best = min(pa.pipe_time(c, **m) for c in _compositions(12, 12))
    got = pa.pipe_time(s, **m)
    assert best <= got <= best * 1.03


def test_invalid_models_and_schedules():
    with pytest.raises(pa.PAError):
        pa.pipe_time([1, 0], **model())
    with pytest.raises(pa.PAError):
        pa.pipe_time([1], **model(n_sets=0))
    with pytest.raises(pa.PAError):
        pa.pipe_time([1], **model(items_per_frame=0))
    with pytest.raises(pa.PAError):
        pa.pipe_schedule(0, 4, **model())
    with pytest.raises(pa.PAError):
        pa.pipe_schedule(4, 0, **model())


def test_long_calls_get_full_middle_chunks():
    """10 000 frames in chunks of at most 32: the search stays quick and
    returns a valid schedule built from full middle chunks."""
    import time

    m = model(items_per_frame=256, resident=608, upload_us=4.9, download_us=16.4,
              kernel_us=25.0, launch_us=30.0, wave_share=0.5)
    t0 = time.perf_counter()
    s = pa.pipe_schedule(10000, 32, **m)
    assert time.perf_counter() - t0 < 5.0
    _valid(s, 10000, 32)
    assert s.count(32) >= 300
