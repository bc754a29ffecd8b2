"""Checkpoint and resume of a streaming context (tpc_snapshot / tpc_restore):
a stream interrupted between two pushes and continued in a new context must
give exactly the labels and features of the uninterrupted stream, i.e. of the
one-shot oracle on the whole stream (Algorithm 3, steps 1 and 9 hand buffers
over between processing steps; no step may change a cluster)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import assert_features_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2412_11809_gb300 import CLUSTER_DTYPE, Clusterer, TpcError  # noqa: E402
from paper_2412_11809_gb300.binding import SNAPSHOT_HEADER_DTYPE, HIT_DTYPE  # noqa: E402


def header(snap: bytes):
    return np.frombuffer(snap[:64], dtype=SNAPSHOT_HEADER_DTYPE)[0]


def push_collect(c, chunks, out):
    for ch in chunks:
        c.push(ch)
        lab, idx = c.labels(with_indices=True)
        out[0].append(idx)
        out[1].append(lab)
        out[2].append(c.features())


def finish(c, out):
    c.flush()
    lab, idx = c.labels(with_indices=True)
    out[0].append(idx)
    out[1].append(lab)
    out[2].append(c.features())
    return (np.concatenate(out[0]), np.concatenate(out[1]),
            np.concatenate(out[2]) if out[2] else np.zeros(0, CLUSTER_DTYPE))


def check(hits, idx, lab, rec, w=256, h=256, dt=128):
    n = len(hits)
    assert len(idx) == n, "every hit finalised exactly once"
    order = np.argsort(idx)
    np.testing.assert_array_equal(idx[order], np.arange(n))
    want = oracle.labels(hits, w, h, dt)
    np.testing.assert_array_equal(lab[order], want)
    rec = rec[np.argsort(rec["label"], kind="stable")]
    assert_features_equal(rec, oracle.features(hits, want))


def split(hits, sizes):
    cuts = np.cumsum(sizes)[:-1]
    return np.split(hits, cuts)


def test_resume_in_new_context_equals_uninterrupted():
    [(hits, sizes, t)] = synth.cfg3(hits_per_stream=1_200_000, n_streams=1, seed=71,
                                    chunk_lo=20_000, chunk_hi=200_000)
    chunks = split(hits, sizes)
    k = len(chunks) // 2
    out = ([], [], [])
    with Clusterer(256, 256, 128, max_disorder=t) as a:
        push_collect(a, chunks[:k], out)
        _, _, n_open = a.counts()
        snap = a.snapshot()
        h = header(snap)
        assert h["magic"] == 0x53435054 and h["version"] == 1
        assert (h["width"], h["height"], h["dt"], h["max_disorder"]) == (256, 256, 128, t)
        assert h["pushed"] == sum(sizes[:k])
        assert h["n_carry"] == n_open > 0
        assert len(snap) == 64 + 24 * n_open
        carried = np.frombuffer(snap[64:64 + 16 * n_open], dtype=HIT_DTYPE)
        gidx = np.frombuffer(snap[64 + 16 * n_open:], dtype=np.uint64)
        # the carry is the pushed hits not yet finalised, with their indices
        assert np.all(gidx < h["pushed"])
        np.testing.assert_array_equal(carried, hits[gidx.astype(np.int64)])
        done = np.concatenate(out[0]) if out[0] else np.zeros(0, np.uint64)
        assert not np.isin(gidx, done).any()
        assert len(done) + n_open == h["pushed"]
        assert h["has_seen"] == 1 and h["seen_max"] == hits["toa"][:h["pushed"]].max()
        # the context itself keeps streaming after a snapshot
        assert a.snapshot() == snap
    with Clusterer(256, 256, 128) as b:          # not streaming yet: restore sets it
        b.restore(snap)
        assert b.snapshot() == snap               # the restored state, byte for byte
        push_collect(b, chunks[k:], out)
        idx, lab, rec = finish(b, out)
    check(hits, idx, lab, rec)


def test_restore_grows_used_context():
    """A context that streamed and flushed before (small carry buffer) takes a
    snapshot with a carry larger than its buffers; an empty snapshot after a
    flush restores too."""
    hits, t = synth.cfg1(scale=600_000 / (64 * 2**20), seed=73)
    wide = 4_000_000   # a large disorder bound: about 250k hits stay open
    n1 = 400_000
    out = ([], [], [])
    with Clusterer(256, 256, 128, max_disorder=wide) as a:
        push_collect(a, [hits[:n1 // 2], hits[n1 // 2:n1]], out)
        snap = a.snapshot()
    assert header(snap)["n_carry"] > 70_000
    other, _ = synth.cfg0(scale=0.01, seed=5)
    with Clusterer(256, 256, 128, max_disorder=1000) as b:
        b.push(other[:2000])
        b.flush()
        b.labels()
        b.restore(snap)
        assert header(b.snapshot())["max_disorder"] == wide
        push_collect(b, [hits[n1:]], out)
        idx, lab, rec = finish(b, out)
        after = b.snapshot()
    check(hits, idx, lab, rec)
    h = header(after)
    assert h["n_carry"] == 0 and h["pushed"] == len(hits)
    with Clusterer(256, 256, 128) as c:          # resume after the end of a stream
        c.restore(after)
        more = hits[:1000].copy()                # a later continuation of the stream
        more["toa"] += hits["toa"].max() + 1_000_000
        c.push(more)                             # indices continue from `pushed`
        c.flush()
        lab, idx = c.labels(with_indices=True)
        np.testing.assert_array_equal(np.sort(idx), len(hits) + np.arange(1000))


def test_restored_watermark_rejects_late_hits():
    hits, t = synth.cfg0(scale=0.05, seed=3)
    hits = hits[np.argsort(hits["toa"], kind="stable")]
    with Clusterer(256, 256, 128, max_disorder=10) as a:
        a.push(hits[: len(hits) // 2])
        snap = a.snapshot()
    with Clusterer(256, 256, 128) as b:
        b.restore(snap)
        with pytest.raises(TpcError) as e:
            b.push(hits[:10].copy())
            b.sync()
        assert e.value.name == "TPC_ERR_LATE"


def test_checkpoint_errors():
    [(hits, sizes, t)] = synth.cfg3(hits_per_stream=200_000, n_streams=1, seed=75,
                                    chunk_lo=20_000, chunk_hi=60_000)
    with Clusterer(256, 256, 128) as plain:
        with pytest.raises(TpcError) as e:
            plain.snapshot()
        assert e.value.name == "TPC_ERR_STATE"
    with Clusterer(256, 256, 128, max_disorder=t) as a:
        a.push(hits[:100_000])
        snap = a.snapshot()
        with pytest.raises(TpcError) as e:      # open hits: a restore would drop them
            a.restore(snap)
        assert e.value.name == "TPC_ERR_STATE"
    assert header(snap)["n_carry"] > 0
    bad_magic = bytearray(snap)
    bad_magic[0] ^= 1
    for blob, what in [(bytes(bad_magic), "magic"), (snap[:-8], "size"), (snap[:32], "short")]:
        with Clusterer(256, 256, 128) as b:
            with pytest.raises(TpcError) as e:
                b.restore(blob)
            assert e.value.name == "TPC_ERR_ARG", what
    for w, h, dt in [(256, 255, 128), (128, 256, 128), (256, 256, 64)]:
        with Clusterer(w, h, dt) as b:
            with pytest.raises(TpcError) as e:
                b.restore(snap)
            assert e.value.name == "TPC_ERR_ARG"
    with Clusterer(256, 256, 128, variant="static") as b:
        with pytest.raises(TpcError) as e:
            b.restore(snap)
        assert e.value.name == "TPC_ERR_ARG"
    with Clusterer(256, 256, 128) as b:          # pending one-shot hits
        b.push(hits[:10].copy())
        with pytest.raises(TpcError) as e:
            b.restore(snap)
        assert e.value.name == "TPC_ERR_STATE"
