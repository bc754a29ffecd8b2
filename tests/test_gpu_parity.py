"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Labels must match bit-exactly; size, sum ToT and first ToA exactly; the fp32
centroids within 1e-5 relative of the fp64 oracle.  Sizes span several tiles
(4096 hits) with ragged tails; edge cases cover empty and single inputs,
degenerate piles on one pixel or one ToA, sensor borders, ToA near 2^64 and
the error paths.
"""
import numpy as np
import pytest

import oracle
import synth
from bruteforce import random_hits
from gpu_helpers import (assert_features_equal, check_against_oracle, run_gpu,
                         sampled_cluster_check)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2412_11809_gb300 import Clusterer, TpcError  # noqa: E402


def test_cfg0_full_size():
    hits, _ = synth.cfg0()
    check_against_oracle(hits, 256, 256, synth.DT_200NS)


def test_cfg1_scaled():
    hits, _ = synth.cfg1(scale=1 / 16)
    check_against_oracle(hits, 256, 256, synth.DT_200NS)


def test_cfg4_timepix4_scaled_both_windows():
    hits, _ = synth.cfg4(scale=1 / 256)
    check_against_oracle(hits, 448, 512, synth.DT_200NS)
    check_against_oracle(hits, 448, 512, synth.DT_600NS)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 4095, 4096, 4097, 8191, 12289, 40000])
def test_ragged_sizes(n):
    rng = np.random.default_rng(n)
    hits = random_hits(rng, n, 40, 30, max(1, n * 3))
    check_against_oracle(hits, 40, 30, 7)


@pytest.mark.parametrize("seed", range(6))
def test_random_dense_small_sensor(seed):
    """Tiny sensors and dense time: long same-pixel chains, halos spanning tiles."""
    rng = np.random.default_rng(100 + seed)
    w, h = int(rng.integers(1, 9)), int(rng.integers(1, 9))
    n = int(rng.integers(5000, 30000))
    hits = random_hits(rng, n, w, h, int(rng.integers(0, 4 * n)))
    check_against_oracle(hits, w, h, int(rng.integers(0, 50)))


def test_pile_on_one_pixel():
    n = 20000
    hits = oracle.make_hits(np.zeros(n, int), np.zeros(n, int), np.arange(n)[::-1] * 3)
    lab, _ = check_against_oracle(hits, 1, 1, 3)
    assert len(np.unique(lab)) == 1
    lab, _ = check_against_oracle(hits, 1, 1, 2)
    assert len(np.unique(lab)) == n


def test_hot_pixel_mixes_table_and_general_tiles():
    """A pixel hit far more often than the table link's list walk allows sends
    the tiles of that burst to the general link kernel while the others stay
    in table mode; clusters joining both kinds of tiles must come out exact."""
    rng = np.random.default_rng(21)
    bg = random_hits(rng, 60000, 64, 64, 120000)
    n_hot = 1500
    hot = oracle.make_hits(np.full(n_hot, 31), np.full(n_hot, 31),
                           np.sort(rng.integers(50000, 56000, n_hot)), rng.integers(1, 20, n_hot))
    hits = np.concatenate([bg, hot])
    hits = hits[np.argsort(hits["toa"], kind="stable")]
    lab, _ = check_against_oracle(hits, 64, 64, 500)
    t_of = np.arange(len(hits)) // 4096
    first = {}
    spans = 0
    for i, l in enumerate(lab):
        if int(l) in first and first[int(l)] != t_of[i]:
            spans += 1
        first.setdefault(int(l), t_of[i])
    assert spans > 100   # many clusters cross tile borders


def test_all_same_toa_is_pixel_ccl():
    rng = np.random.default_rng(7)
    hits = random_hits(rng, 30000, 200, 150, 0)
    hits["toa"] = 123456789
    check_against_oracle(hits, 200, 150, 0)


def test_borders_and_corners():
    rng = np.random.default_rng(8)
    W, H = 64, 48
    xs = rng.choice([0, 1, W - 2, W - 1], 20000)
    ys = rng.choice([0, 1, H - 2, H - 1], 20000)
    hits = oracle.make_hits(xs, ys, rng.integers(0, 200000, 20000), rng.integers(1, 100, 20000))
    check_against_oracle(hits, W, H, 10)


def test_toa_near_top_of_range():
    rng = np.random.default_rng(9)
    hits = random_hits(rng, 10000, 32, 32, 50000)
    hits["toa"] += np.uint64(2**64 - 60000)
    check_against_oracle(hits, 32, 32, 20)


def test_dt_zero_and_huge():
    hits, _ = synth.cfg0(scale=0.02, seed=3)
    check_against_oracle(hits, 256, 256, 0)
    check_against_oracle(hits, 256, 256, 2**40)


def test_host_push_and_multiple_pushes():
    hits, _ = synth.cfg0(scale=0.05, seed=4)
    want = oracle.labels(hits, 256, 256, 128)
    for device, pushes in ((False, 1), (False, 3), (True, 5)):
        lab, feats = run_gpu(hits, 256, 256, 128, device=device, pushes=pushes)
        np.testing.assert_array_equal(lab, want)


def test_input_permutation():
    hits, _ = synth.cfg1(scale=1 / 256, seed=5)
    perm = np.random.default_rng(0).permutation(len(hits))
    check_against_oracle(hits[perm], 256, 256, 128)


@pytest.mark.parametrize("window", [2400, 5000])
def test_wide_disorder_merge_windows(window):
    """Streams shuffled over wider windows than the bench stream's 1000
    positions: at 2400 the sorted tiles of every border interleave over more
    than the merge's first band (1024 positions on each side; about 1200
    here), so the borders are merged over the whole window (2048 on each
    side); at 5000 they interleave over about 2400 and the step takes the
    general radix sort.
    Both must give the oracle's clusters (t-ordered input, Section 3.1)."""
    hits, _ = synth.generate(256, 256, 600_000, 40 + window, hit_rate_hz=40e6, track_frac=0.2,
                             dead_time=True, shuffle_window=window)
    check_against_oracle(hits, 256, 256, synth.DT_200NS)


def test_empty_flush():
    with Clusterer(256, 256, 128) as c:
        c.flush()
        assert c.counts() == (0, 0, 0)
        assert len(c.labels()) == 0 and len(c.features()) == 0


def test_out_of_range_reported():
    hits = oracle.make_hits([1, 300], [1, 1], [5, 6])
    with Clusterer(256, 256, 128) as c:
        c.push(hits)
        c.flush()
        with pytest.raises(TpcError) as e:
            c.sync()
        assert e.value.name == "TPC_ERR_RANGE"


def test_far_out_of_range_reported():
    """Coordinates far outside the sensor: reported, and the per-pixel tables
    of the link kernels are never indexed with them (pixels are clamped)."""
    hits = oracle.make_hits([1, 65535, 3, 40000], [1, 65535, 2, 7], [5, 6, 7, 8])
    for w, h in ((256, 256), (1024, 1024)):
        with Clusterer(w, h, 128) as c:
            c.push(hits)
            c.flush()
            with pytest.raises(TpcError) as e:
                c.sync()
            assert e.value.name == "TPC_ERR_RANGE"


def test_span_too_large_reported():
    hits = oracle.make_hits([1, 2], [1, 1], [0, 2**33])
    with Clusterer(256, 256, 128) as c:
        c.push(hits)
        c.flush()
        with pytest.raises(TpcError) as e:
            c.sync()
        assert e.value.name == "TPC_ERR_SPAN"


def test_bad_arguments():
    with pytest.raises(TpcError):
        Clusterer(0, 256, 128)
    with pytest.raises(TpcError):
        Clusterer(4096, 4096, 128)   # more than 2^20 pixels
    with pytest.raises(KeyError):
        Clusterer(256, 256, 128, "nonsense")


def test_repeat_flushes_continue_global_indices():
    a, _ = synth.cfg0(scale=0.01, seed=11)
    b, _ = synth.cfg0(scale=0.01, seed=12)
    with Clusterer(256, 256, 128) as c:
        c.push(a)
        c.flush()
        la = c.labels()
        c.push(b)
        c.flush()
        lb, ib = c.labels(with_indices=True)
    np.testing.assert_array_equal(la, oracle.labels(a, 256, 256, 128))
    np.testing.assert_array_equal(ib, np.arange(len(a), len(a) + len(b)))
    np.testing.assert_array_equal(lb, oracle.labels(b, 256, 256, 128) + len(a))


@pytest.mark.slow
def test_cfg1_full_size_sampled():
    """The benchmark workload at full size (64M hits), in the launch
    configuration the benchmark uses; exact checks of sampled clusters plus
    properties that hold at any size."""
    hits, _ = synth.cfg1()
    dev = torch.from_numpy(hits.view(np.uint8).reshape(-1, 16)).cuda()
    with Clusterer(256, 256, synth.DT_200NS) as c:
        c.push(dev)
        c.flush()
        lab = c.labels()
        feats = c.features()
    n = len(hits)
    idx = np.arange(n, dtype=np.uint64)
    assert np.all(lab <= idx)
    assert np.all(lab[lab.astype(np.int64)] == lab)
    assert feats["size"].sum() == n
    assert feats["sum_tot"].sum() == hits["tot"].astype(np.int64).sum()
    np.testing.assert_array_equal(feats["label"], np.unique(lab))
    checked = sampled_cluster_check(hits, lab, 256, 256, synth.DT_200NS, 150,
                                    np.random.default_rng(1))
    assert checked > 50
    # every label and record against the paper's temporal-split CPU method
    # (cpu_baseline, itself bit-exact against the oracle in the CPU suite),
    # which clusters the whole stream in a few seconds on the host cores
    import os
    import cpu_baseline
    want, rec, _ = cpu_baseline.cluster(hits, 256, 256, synth.DT_200NS, 6400, max(1, len(os.sched_getaffinity(0))))
    np.testing.assert_array_equal(lab, want)
    assert_features_equal(feats, rec)


def test_labels_async_and_two_context_pipeline():
    """Queued label copies (tpc_labels_async) equal the synchronous ones, also
    when two contexts on two CUDA streams take steps in turn and one step's
    copies overlap the other's kernels."""
    hits, _ = synth.cfg0(scale=0.05, seed=9)
    n = len(hits)
    want = oracle.labels(hits, 256, 256, 128)
    want_rec = oracle.features(hits, want)
    pin_in = torch.from_numpy(hits.view(np.uint8).reshape(-1, 16)).pin_memory()
    ctxs = [Clusterer(256, 256, 128, stream=torch.cuda.Stream()) for _ in range(2)]
    bufs = [torch.empty(n, dtype=torch.int64).pin_memory() for _ in ctxs]
    def shifted(rec, base):   # labels are global indices: a context's k-th step adds k * n
        rec = rec.copy()
        rec["label"] += base
        return rec

    try:
        for step in range(4):
            c = ctxs[step % 2]
            c.push_ptr(pin_in.data_ptr(), n, device=False)
            c.flush()
            assert c.labels_async(bufs[step % 2].data_ptr(), n, device=False) == n
            if step:
                prev, base = ctxs[(step - 1) % 2], n * ((step - 1) // 2)
                assert_features_equal(prev.features(), shifted(want_rec, base))   # waits for that step
                np.testing.assert_array_equal(bufs[(step - 1) % 2].numpy(), want + base)
        ctxs[1].sync()
        np.testing.assert_array_equal(bufs[1].numpy(), want + n)
        with pytest.raises(TpcError) as e:
            ctxs[0].labels_async(bufs[0].data_ptr(), n - 1, device=False)
        assert e.value.name == "TPC_ERR_CAP"
    finally:
        for c in ctxs:
            c.close()
    with Clusterer(256, 256, 128, max_disorder=10**6) as c:
        c.push(hits[:1000])
        with pytest.raises(TpcError) as e:
            c.labels_async(bufs[0].data_ptr(), n, device=False)
        assert e.value.name == "TPC_ERR_STATE"


@pytest.mark.parametrize("w,h,seed", [(300, 600, 31), (301, 500, 32), (4000, 200, 33), (1024, 1024, 34)])
def test_banded_table_sensors(w, h, seed):
    """Sensors larger than the shared-memory pixel table are linked band by
    band (rows of the table); clusters crossing band edges, odd widths and
    thin bands (a wide sensor) must come out exact."""
    rng = np.random.default_rng(seed)
    n = 60000
    hits = random_hits(rng, n, w, h, n // 2)
    # dense vertical tracks so that many clusters cross band edges
    ys = np.arange(h)
    tracks = []
    for x in rng.integers(1, w - 1, 8):
        t0 = int(rng.integers(0, n // 2))
        tracks.append(oracle.make_hits(np.full(h, x), ys, t0 + (ys % 7), rng.integers(1, 30, h)))
    hits = np.concatenate([hits] + tracks)
    hits = hits[np.argsort(hits["toa"], kind="stable")]
    check_against_oracle(hits, w, h, 64)


def test_wide_span_takes_general_sort():
    """A step whose ToA span reaches past 2^31 ticks from its first hit (but
    stays under 2^32) leaves the tile sort's keys out of range; the general
    sort takes over and the result is still exact."""
    rng = np.random.default_rng(5)
    hits = random_hits(rng, 20000, 64, 64, 3_500_000_000)
    hits = hits[np.argsort(hits["toa"], kind="stable")]
    lab, _ = check_against_oracle(hits, 64, 64, 200_000_000)
    assert len(np.unique(lab)) < len(hits)   # clusters did form


@pytest.mark.parametrize("cap", [1, 2])
def test_cta_cap_gives_the_same_result(cap):
    """TPC_OPT_CTAS_PER_SM caps every persistent grid below its occupancy;
    each kernel loops over its tiles whatever the grid, so labels and
    features are unchanged (one-shot (a), and variant (c))."""
    hits, _ = synth.cfg1(scale=1_500_000 / (64 * 2**20), seed=95)
    check_against_oracle(hits, 256, 256, 128, ctas_per_sm=cap)
    check_against_oracle(hits[:200_000], 256, 256, 128, "static", ctas_per_sm=cap)


@pytest.mark.parametrize("variant", ["local", "static", "global"])
def test_bound_outputs_written_in_place(variant):
    """tpc_bind_outputs: the step writes labels and records straight into the
    caller's device buffers, equal to the oracle's; retrieval still works;
    too small a buffer refuses the step and leaves the hits pending."""
    from paper_2412_11809_gb300 import CLUSTER_DTYPE
    hits, _ = synth.cfg1(scale=1 / 256, seed=71)
    n = len(hits)
    want = oracle.labels(hits, 256, 256, 128, variant)
    ref = oracle.features(hits, want)
    d_lab = torch.full((n,), -1, dtype=torch.int64, device="cuda")
    d_rec = torch.zeros((n, CLUSTER_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
    with Clusterer(256, 256, 128, variant) as c:
        c.bind_outputs(d_lab.data_ptr(), d_rec.data_ptr(), n)
        for rep in range(2):
            c.push(torch.from_numpy(hits.view(np.uint8).reshape(-1, 16)).cuda())
            c.flush()
            _, m, _ = c.counts()
            np.testing.assert_array_equal(d_lab.cpu().numpy().view(np.uint64) - np.uint64(rep * n), want)
            rec = d_rec.cpu().numpy().view(CLUSTER_DTYPE).reshape(-1)[:m].copy()
            rec["label"] -= np.uint64(rep * n)
            assert_features_equal(rec, ref)
            np.testing.assert_array_equal(c.labels() - np.uint64(rep * n), want)   # retrieval copies too
        small = torch.zeros((n // 2, CLUSTER_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
        c.bind_outputs(d_lab.data_ptr(), small.data_ptr(), n // 2)
        c.push(hits)
        with pytest.raises(TpcError) as e:
            c.flush()
        assert e.value.name == "TPC_ERR_CAP"
        c.bind_outputs(None, None)
        c.flush()                                  # the hits were left pending
        np.testing.assert_array_equal(c.labels() - np.uint64(2 * n), want)
    with Clusterer(256, 256, 128) as c:
        host = np.zeros(n, dtype=np.uint64)
        with pytest.raises(TpcError):
            c.bind_outputs(host.ctypes.data, host.ctypes.data, n)
