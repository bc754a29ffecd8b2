"""The temporal-split parallel CPU baseline (paper, Sections 3.2-3.3; a
comparison for the benchmark, not the product) equals the oracle exactly:
labels bit-exact and records identical (its centroids are the same fp64
divisions of exact integer sums), for any window width above dt and any
thread count, including clusters that span many windows."""
import numpy as np
import pytest

import cpu_baseline
import oracle
import synth


def same(hits, w, h, dt, window, threads):
    lab, rec, casc = cpu_baseline.cluster(hits, w, h, dt, window, threads)
    want = oracle.labels(hits, w, h, dt)
    np.testing.assert_array_equal(lab, want)
    ref = oracle.features(hits, want)
    assert len(rec) == len(ref)
    for k in ("label", "size", "sum_tot", "first_toa"):
        np.testing.assert_array_equal(rec[k], ref[k])
    for k in ("cx", "cy"):
        np.testing.assert_array_equal(rec[k], ref[k])
    return casc


@pytest.fixture(scope="module")
def cfg1_small():
    return synth.cfg1(scale=300_000 / (64 * 2**20), seed=5)


@pytest.mark.parametrize("window,threads", [(6400, 1), (6400, 4), (200, 3), (129, 7),
                                            (10**9, 2), (70_000, 5), (1000, 16)])
def test_equals_oracle_cfg1(cfg1_small, window, threads):
    hits, _ = cfg1_small
    casc = same(hits, 256, 256, 128, window, threads)
    # the cascade's counters add up: every pair examined is cut by one of the
    # two cheap tests, merged, or rejected by the full check
    assert casc["cut_by_time"] + casc["cut_by_box"] + casc["merged"] <= casc["pairs"]
    if window < 10**9:
        assert casc["merged"] > 0            # clusters really cross window borders


def test_equals_oracle_large_sensor():
    hits, _ = synth.cfg4(scale=200_000 / (512 * 2**20), seed=6)
    for dt in (128, 384):
        same(hits, 448, 512, dt, 4 * dt, 6)


def test_track_spanning_many_windows():
    """A slow track crosses dozens of windows: the merges chain through every
    border (a cluster of one window merges on both of its sides)."""
    n = 300
    x = np.arange(n) % 256
    y = np.arange(n) // 256 * 2
    toa = 1000 + np.arange(n, dtype=np.uint64) * 100          # 100 ticks per pixel
    rng = np.random.default_rng(1)
    bx, by = rng.integers(0, 256, 500), rng.integers(100, 256, 500)
    btoa = rng.integers(1000, 1000 + 100 * n, 500).astype(np.uint64)
    hits = oracle.make_hits(np.r_[x, bx], np.r_[y, by], np.r_[toa, btoa], np.r_[np.full(n, 3), np.full(500, 2)])
    perm = rng.permutation(len(hits))
    casc = same(hits[perm], 256, 256, 128, 129, 2)
    # 800 hits on 2 workers allow at most 800 / 4 + 1 windows (sparse input
    # widens them): about 200 borders, each crossed by the track
    assert casc["merged"] >= 150


def test_edges():
    e = np.zeros(0, dtype=oracle.HIT_DTYPE)
    lab, rec, _ = cpu_baseline.cluster(e, 256, 256, 128, 6400, 4)
    assert len(lab) == 0 and len(rec) == 0
    one = oracle.make_hits([3], [4], [77])
    same(one, 256, 256, 128, 6400, 8)                      # more threads than hits
    flat = oracle.make_hits(np.arange(64) % 8, np.arange(64) // 8, np.full(64, 500))
    same(flat, 8, 8, 0, 1, 3)                              # one ToA, dt = 0
    # hits on both sides of a border, exactly dt apart (inclusive) and dt + 1
    b = 1000 + 6400
    pair = oracle.make_hits([5, 6, 20, 21], [5, 5, 9, 9], [b - 64, b + 64, b - 64, b + 65])
    lab, _, _ = cpu_baseline.cluster(pair, 256, 256, 128, 6400, 2)
    np.testing.assert_array_equal(lab, oracle.labels(pair, 256, 256, 128))
    assert lab[1] == 0 and lab[3] == 3


def test_toa_near_top_of_range():
    """ToAs within 2^20 ticks of 2^64 and a wide dt: the border slabs are
    found by differences, nothing wraps."""
    rng = np.random.default_rng(12)
    n = 30_000
    toa = np.uint64(2**64 - 2**20) + rng.integers(0, 2**20 - 1, n).astype(np.uint64)
    hits = oracle.make_hits(rng.integers(0, 32, n), rng.integers(0, 32, n), toa, rng.integers(1, 50, n))
    for dt, window in ((20, 200), (5000, 5001), (2**62, 2**62 + 1)):
        same(hits, 32, 32, dt, window, 3)


def test_arguments():
    h = oracle.make_hits([300], [0], [5])
    with pytest.raises(ValueError, match="outside"):
        cpu_baseline.cluster(h, 256, 256, 128, 6400, 2)
    h = oracle.make_hits([1], [0], [5])
    for window in (128, 5):
        with pytest.raises(ValueError, match="argument"):
            cpu_baseline.cluster(h, 256, 256, 128, window, 2)
