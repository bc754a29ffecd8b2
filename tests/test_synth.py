"""The seeded input generator: determinism, ranges, the t-ordered property it
reports (Section 3.1's definition), and the workload shapes it stands in for."""
import numpy as np

import synth


def test_deterministic_and_in_range():
    a, ta = synth.cfg1(scale=1 / 256, seed=42)
    b, tb = synth.cfg1(scale=1 / 256, seed=42)
    assert ta == tb and np.array_equal(a, b)
    c, _ = synth.cfg1(scale=1 / 256, seed=43)
    assert not np.array_equal(a, c)
    assert a["x"].max() < 256 and a["y"].max() < 256
    assert a["tot"].min() >= 1 and a["tot"].max() <= 1023
    assert np.all(a["reserved"] == 0)


def test_reported_disorder_is_tight():
    h, t = synth.cfg0(scale=0.05, seed=1)
    toa = h["toa"].astype(np.int64)
    run_max = np.maximum.accumulate(toa)
    inversion = (run_max[:-1] - toa[1:]).max()
    assert t == max(1, inversion + 1)
    # t-ordered: toa[i] < toa[j] + t for all i < j
    assert np.all(run_max[:-1] < toa[1:] + t)


def test_window_shuffle_displacement():
    h, _ = synth.generate(64, 64, 20000, 9, event_rate_hz=1e6, shuffle_window=1000)
    order = np.argsort(h["toa"], kind="stable")
    disp = np.abs(order - np.arange(len(h)))
    assert 0 < disp.max() < 2000


def test_multi_detector_and_serving_shapes():
    dets = synth.cfg2(scale=1 / 512, seed=5)
    assert len(dets) == 16
    assert [d[:2] for d in dets] == [(256, 256)] * 10 + [(448, 512)] * 6
    for w, h, hits, sizes, t in dets:
        assert len(hits) == sum(sizes)
    streams = synth.cfg3(hits_per_stream=200_000, n_streams=3, seed=1)
    for hits, sizes, t in streams:
        assert sum(sizes) == len(hits) and all(s >= 65536 for s in sizes[:-1])


def test_recipe_statistics():
    """The generator draws what the input recipe states: ToT = min(1023,
    1 + round(Exp(40))); blobs of 1 + Geometric(0.3) distinct pixels (mean
    1 + 0.7/0.3 = 3.33) at 1 Mevent/s; a hit rate of 40 Mhits/s for config 1
    (1 tick = 1.5625 ns)."""
    import oracle
    a, _ = synth.generate(256, 256, 400_000, 17, event_rate_hz=1e6, shuffle_window=1)
    tot = a["tot"].astype(np.float64)
    assert abs(tot.mean() - 41.0) < 0.5                    # 1 + E[round(Exp(40))] ~ 41
    assert a["tot"].min() == 1 and a["tot"].max() <= 1023
    # blobs at 1 Mevent/s on 65536 pixels almost never touch: clusters = blobs
    lab = oracle.labels(a, 256, 256, 128)
    sizes = np.bincount(np.unique(lab, return_inverse=True)[1])
    assert abs(sizes.mean() - (1 + 0.7 / 0.3)) < 0.1
    span_s = (int(a["toa"].max()) - int(a["toa"].min())) * 1.5625e-9
    assert abs(len(sizes) / span_s / 1e6 - 1.0) < 0.05     # events per second
    h, _ = synth.cfg1(scale=1 / 64, seed=3)
    span_s = (int(h["toa"].max()) - int(h["toa"].min())) * 1.5625e-9
    assert abs(len(h) / span_s / 40e6 - 1.0) < 0.05        # hits per second


def test_blocked_generation_is_one_t_ordered_stream():
    """The full-size 448x512 stream is drawn as consecutive sub-streams in
    parallel: deterministic, t-ordered with the reported t, blocks in time
    order with a quiet gap longer than any ToT between them."""
    a, ta = synth.cfg4(scale=1 / 2048, seed=7, blocks=4)
    b, tb = synth.cfg4(scale=1 / 2048, seed=7, blocks=4)
    assert ta == tb and np.array_equal(a, b)
    assert len(a) == 512 * 2**20 // 2048
    toa = a["toa"].astype(np.int64)
    run_max = np.maximum.accumulate(toa)
    assert ta == max(1, int((run_max[:-1] - toa[1:]).max()) + 1)
    sizes = [len(a) // 4] * 4
    edges = np.cumsum(sizes)[:-1]
    for e in edges:   # every hit of a block precedes every hit of the next
        assert toa[:e].max() + 1024 < toa[e:].min()
    assert a["x"].max() < 448 and a["y"].max() < 512 and a["tot"].max() <= 1023
