"""Streaming with device-resident open clusters (chunks cut at arbitrary
points), concurrent streams, admission by memory budget, late-hit detection,
and the batched multi-detector step — each against the one-shot oracle on the
concatenated stream (the paper's merging of border/open clusters, Section
3.3, and hit buffering, Algorithm 2, must not change any cluster)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import assert_features_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2412_11809_gb300 import CLUSTER_DTYPE, Clusterer, TpcError, batch_flush  # noqa: E402


def collect_stream(c, hits, sizes):
    """Push chunks, gather every finalised (index, label) and record."""
    idx_all, lab_all, rec_all = [], [], []
    start = 0
    for s in sizes:
        c.push(hits[start:start + s])
        start += s
        lab, idx = c.labels(with_indices=True)
        idx_all.append(idx)
        lab_all.append(lab)
        rec_all.append(c.features())
    c.flush()
    lab, idx = c.labels(with_indices=True)
    idx_all.append(idx)
    lab_all.append(lab)
    rec_all.append(c.features())
    return (np.concatenate(idx_all), np.concatenate(lab_all),
            np.concatenate(rec_all) if rec_all else np.zeros(0, CLUSTER_DTYPE))


def check_stream_result(hits, idx, lab, rec, w=256, h=256, dt=128):
    n = len(hits)
    assert len(idx) == n, "every hit finalised exactly once"
    order = np.argsort(idx)
    np.testing.assert_array_equal(idx[order], np.arange(n))
    want = oracle.labels(hits, w, h, dt)
    np.testing.assert_array_equal(lab[order], want)
    rec = rec[np.argsort(rec["label"], kind="stable")]
    assert_features_equal(rec, oracle.features(hits, want))
    return want


def straddle_fraction(labels, sizes):
    chunk_of = np.repeat(np.arange(len(sizes)), sizes)
    first = {}
    straddle = set()
    for i, l in enumerate(labels):
        l = int(l)
        if l in first and first[l] != chunk_of[i]:
            straddle.add(l)
        first.setdefault(l, chunk_of[i])
    return len(straddle) / max(1, len(first))


def test_streaming_equals_one_shot():
    [(hits, sizes, t)] = synth.cfg3(hits_per_stream=1_500_000, n_streams=1, seed=41,
                                    chunk_lo=20_000, chunk_hi=300_000)
    with Clusterer(256, 256, 128, max_disorder=t) as c:
        idx, lab, rec = collect_stream(c, hits, sizes)
    want = check_stream_result(hits, idx, lab, rec)
    assert straddle_fraction(want, sizes) > 0     # the cut really splits clusters


def test_streaming_tiny_chunks_and_carry_growth():
    """Chunks far smaller than a cluster's time span: most hits are carried
    several steps; the carry buffer has to grow."""
    hits, t = synth.cfg1(scale=200_000 / (64 * 2**20), seed=43)
    rng = np.random.default_rng(0)
    sizes = []
    left = len(hits)
    while left:
        s = int(min(left, rng.integers(1, 3000)))
        sizes.append(s)
        left -= s
    with Clusterer(256, 256, 128, max_disorder=t) as c:
        idx, lab, rec = collect_stream(c, hits, sizes)
    check_stream_result(hits, idx, lab, rec)


def test_concurrent_streams_same_alone_and_in_mix():
    streams = synth.cfg3(hits_per_stream=400_000, n_streams=4, seed=47,
                         chunk_lo=20_000, chunk_hi=150_000)
    alone = []
    for hits, sizes, t in streams:
        with Clusterer(256, 256, 128, max_disorder=t) as c:
            alone.append(collect_stream(c, hits, sizes))
    # in the mix: every context on its own CUDA stream, pushes interleaved
    ctxs = [Clusterer(256, 256, 128, max_disorder=t, stream=torch.cuda.Stream())
            for _, _, t in streams]
    got = [([], [], []) for _ in streams]
    pos = [0] * len(streams)
    step = [0] * len(streams)
    live = set(range(len(streams)))
    while live:
        for s in sorted(live):
            hits, sizes, _ = streams[s]
            if step[s] < len(sizes):
                n = sizes[step[s]]
                ctxs[s].push(hits[pos[s]:pos[s] + n])
                pos[s] += n
                step[s] += 1
            else:
                ctxs[s].flush()
                live.discard(s)
            lab, idx = ctxs[s].labels(with_indices=True)
            got[s][0].append(idx)
            got[s][1].append(lab)
            got[s][2].append(ctxs[s].features())
    for c in ctxs:
        c.close()
    for s, (hits, sizes, _) in enumerate(streams):
        idx, lab, rec = (np.concatenate(x) for x in got[s])
        check_stream_result(hits, idx, lab, rec)
        a_idx, a_lab, _ = alone[s]
        np.testing.assert_array_equal(np.sort(idx), np.sort(a_idx))
        np.testing.assert_array_equal(lab[np.argsort(idx)], a_lab[np.argsort(a_idx)])


def test_late_hit_reported():
    hits, t = synth.cfg0(scale=0.05, seed=3)
    hits = hits[np.argsort(hits["toa"], kind="stable")]
    with Clusterer(256, 256, 128, max_disorder=10) as c:
        c.push(hits[: len(hits) // 2])
        late = hits[:10].copy()          # far older than the watermark allows
        with pytest.raises(TpcError) as e:
            c.push(late)
            c.sync()
        assert e.value.name == "TPC_ERR_LATE"


def test_admission_refused_over_budget():
    hits, t = synth.cfg0(scale=0.2, seed=5)
    with Clusterer(256, 256, 128, max_disorder=t, mem_budget=1 << 20) as c:
        with pytest.raises(TpcError) as e:
            c.push(hits)
        assert e.value.name == "TPC_ERR_BUSY"


def test_batched_detectors_equal_single():
    dets = synth.cfg2(scale=1 / 64, seed=7)
    ctxs = [Clusterer(w, h, 128) for w, h, _, _, _ in dets]
    for c, (w, h, hits, sizes, _) in zip(ctxs, dets):
        start = 0
        for s in sizes:                  # several chunks per detector
            c.push(torch.from_numpy(hits[start:start + s].view(np.uint8).reshape(-1, 16)).cuda())
            start += s
    batch_flush(ctxs)
    for c, (w, h, hits, _, _) in zip(ctxs, dets):
        lab = c.labels()
        want = oracle.labels(hits, w, h, 128)
        np.testing.assert_array_equal(lab, want)
        assert_features_equal(c.features(), oracle.features(hits, want))
        c.close()


def test_batched_repeat_and_mixed_sizes():
    """The batch graph is replayed across batches of different sizes."""
    for seed in (11, 12):
        dets = synth.cfg2(scale=1 / 256, seed=seed)
        ctxs = [Clusterer(w, h, 128) for w, h, _, _, _ in dets]
        for c, (_, _, hits, _, _) in zip(ctxs, dets):
            c.push(hits)
        batch_flush(ctxs)
        for c, (w, h, hits, _, _) in zip(ctxs, dets):
            np.testing.assert_array_equal(c.labels(), oracle.labels(hits, w, h, 128))
            c.close()


def test_streaming_large_sensor_banded():
    """Streaming on a sensor larger than the shared-memory pixel table (linked
    band by band), chunks cut at arbitrary points."""
    hits, t = synth.cfg4(scale=600_000 / (512 * 2**20), seed=45)
    rng = np.random.default_rng(1)
    sizes, left = [], len(hits)
    while left:
        s = int(min(left, rng.integers(5_000, 120_000)))
        sizes.append(s)
        left -= s
    with Clusterer(448, 512, 128, max_disorder=t) as c:
        idx, lab, rec = collect_stream(c, hits, sizes)
    check_stream_result(hits, idx, lab, rec, w=448, h=512, dt=128)
