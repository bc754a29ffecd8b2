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
