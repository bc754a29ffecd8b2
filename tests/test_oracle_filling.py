"""Pins of the oracle's hit buffer filling (Algorithm 2, Section 4.1) against
what the paper fixes: a hand-worked example of the procedure, and the
properties Section 4.1 states for it — on a t-ordered stream (Section 3.1)
the buffers are cut at the recorded closing times, so no cluster is split by
unsortedness, and the buffers sent one after another form a t-ordered stream
again (so a streaming consumer can take them in order)."""
import os

import numpy as np
import pytest

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURE = os.path.join(HERE, "golden", "buffer_filling", "worked_example.txt")
END = np.uint64(2**64 - 1)


def load_fixture(path):
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.lstrip().startswith("#")]
    b, b_t, t, t_closing = (int(v) for v in rows[0])
    d = {r[0]: r[1:] for r in rows[1:]}
    toa = np.array([int(v) for v in d["toa"]], dtype=np.uint64)
    buf = np.array([int(v) for v in d["buffer"]], dtype=np.uint64)
    cut = np.array([END if v == "-" else int(v) for v in d["cut"]], dtype=np.uint64)
    hits = oracle.make_hits(np.zeros(len(toa), int), np.zeros(len(toa), int), toa)
    return hits, (b, b_t, t, t_closing), buf, cut


def concat_order(buffer_of):
    """Hit indices in the order the buffers are sent (arrival order inside)."""
    return np.lexsort((np.arange(len(buffer_of)), buffer_of))


def is_t_ordered(toa, t):
    """toa_i < toa_j + t for every i < j  <=>  running max < toa_j + t."""
    toa = toa.astype(np.int64)
    run = np.maximum.accumulate(toa)
    return bool(np.all(run[:-1] < toa[1:] + t))


def test_worked_example():
    hits, params, buf, cut = load_fixture(FIXTURE)
    got_buf, got_cut = oracle.fill_buffers(hits, *params)
    np.testing.assert_array_equal(got_buf, buf)
    np.testing.assert_array_equal(got_cut, cut)


def test_empty_stream_and_bad_arguments():
    e = np.zeros(0, dtype=oracle.HIT_DTYPE)
    buf, cut = oracle.fill_buffers(e, 10, 2, 5, 1)
    assert len(buf) == 0 and len(cut) == 0
    h = oracle.make_hits([0], [0], [5])
    for b, b_t in [(0, 0), (4, 4), (4, 5)]:
        with pytest.raises(ValueError):
            oracle.fill_buffers(h, b, b_t, 5, 1)


def test_sorted_stream_fills_whole_buffers():
    """A sorted stream with t_closing = 0 and b_t = 0 is cut into consecutive
    blocks of b hits, each sent by the first hit more than t after its last."""
    toa = np.arange(0, 1000, dtype=np.uint64) * 10
    h = oracle.make_hits(np.zeros(1000, int), np.zeros(1000, int), toa)
    buf, cut = oracle.fill_buffers(h, 100, 0, 5, 0)
    np.testing.assert_array_equal(buf, np.arange(1000) // 100)
    np.testing.assert_array_equal(cut[:-1], toa[99:999:100])
    assert cut[-1] == END


@pytest.mark.parametrize("seed", [11, 12])
def test_clean_time_cuts_on_t_ordered_stream(seed):
    """Section 4.1: with room b_t for the hits of the closing window, every hit
    of buffer k is earlier than its cut and every hit of a later buffer is at
    or after it; the partition is a cut in time."""
    hits, t = synth.cfg1(scale=300_000 / (64 * 2**20), seed=seed)
    assert is_t_ordered(hits["toa"], t)
    b, b_t, t_closing = 40_000, 12_000, 200
    buf, cut = oracle.fill_buffers(hits, b, b_t, t, t_closing)
    nb = len(cut)
    assert nb >= 5
    counts = np.bincount(buf.astype(np.int64), minlength=nb)
    assert counts.sum() == len(hits) and np.all(counts > 0) and np.all(counts <= b)
    toa = hits["toa"]
    lo = np.array([toa[buf == k].min() for k in range(nb)])
    hi = np.array([toa[buf == k].max() for k in range(nb)])
    for k in range(nb - 1):
        assert hi[k] < cut[k], k
        assert lo[k + 1:].min() >= cut[k], k
    assert np.all(np.diff(cut[:-1].astype(np.int64)) > 0)


@pytest.mark.parametrize("b,b_t,t_closing", [(3000, 100, 0), (5000, 200, 50), (800, 700, 20)])
def test_sent_buffers_stay_t_ordered(b, b_t, t_closing):
    """Even when buffers overflow their room, the buffers sent one after
    another are t-ordered: a hit sent earlier was either received earlier, or
    is earlier than the cut that put the later one into a later buffer.  (With
    too little room a buffer may also start with more than b hits: the next
    buffer has no bound in the procedure.)"""
    hits, t = synth.cfg1(scale=200_000 / (64 * 2**20), seed=13)
    buf, cut = oracle.fill_buffers(hits, b, b_t, t, t_closing)
    order = concat_order(buf)
    assert is_t_ordered(hits["toa"][order], t)
    counts = np.bincount(buf.astype(np.int64))
    assert counts.sum() == len(hits) and np.all(counts > 0) and len(counts) == len(cut)
    # buffers are numbered in the order they are sent: a hit never lands more
    # than one buffer ahead of the current one
    assert np.all(np.diff(np.maximum.accumulate(buf.astype(np.int64))) <= 1)


def test_clusters_split_only_at_cuts():
    """Section 4.1: what Algorithm 2 leaves to border checking is the dt
    neighbourhood of each cut.  Every cluster of the whole stream that the
    buffers split has hits on both sides of a cut within dt of it."""
    hits, t = synth.cfg1(scale=150_000 / (64 * 2**20), seed=14)
    dt = 128
    buf, cut = oracle.fill_buffers(hits, 20_000, 8_000, t, 100)
    lab = oracle.labels(hits, 256, 256, dt)
    toa = hits["toa"].astype(np.int64)
    split = 0
    for l in np.unique(lab):
        members = np.nonzero(lab == l)[0]
        ks = np.unique(buf[members])
        if len(ks) == 1:
            continue
        split += 1
        assert len(ks) == 2 and ks[1] == ks[0] + 1
        c = int(cut[int(ks[0])])
        before = toa[members[buf[members] == ks[0]]]
        after = toa[members[buf[members] == ks[1]]]
        assert before.max() < c <= after.min()
        assert after.min() - before.max() <= dt
    assert split > 0                 # the stream really has clusters across cuts
