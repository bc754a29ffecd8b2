"""The device's union-find forest after a step (tpc_forest), checked on the
host against the invariants of Section 4.1 and against the oracle: every
parent precedes its child in (ToA, input) order, so toa(parent(h)) <= toa(h)
(the paper's time invariant) and each root is its cluster's earliest hit;
every chain ends at a root; the trees are exactly the oracle's clusters."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2412_11809_gb300 import Clusterer, TpcError, batch_flush  # noqa: E402


def roots_of(parent):
    """Follow every chain to its root; returns (root per position, max depth)."""
    cur = parent.astype(np.int64)
    depth = 0
    while True:
        nxt = cur[cur]
        if np.array_equal(nxt, cur):
            return cur, depth
        cur = nxt
        depth += 1
        assert depth < 64, "a chain does not end"


def check_forest(hits, parent, pos, labels_want):
    n = len(hits)
    assert len(parent) == n and len(pos) == n
    np.testing.assert_array_equal(np.sort(pos), np.arange(n))        # a permutation
    toa = hits["toa"][pos]
    assert np.all(np.diff(toa.astype(np.int64)) >= 0)                 # ToA order
    p = parent.astype(np.int64)
    assert np.all(p <= np.arange(n)), "a parent after its child"
    assert np.all(toa[p] <= toa), "time invariant broken"
    root, _ = roots_of(parent)
    # root = the earliest position of its tree
    first = np.full(n, n, np.int64)
    np.minimum.at(first, root, np.arange(n))
    np.testing.assert_array_equal(first[root], root)
    # trees = the oracle's clusters: smallest input index per tree
    best = np.full(n, n, np.int64)
    np.minimum.at(best, root, pos.astype(np.int64))
    got = np.empty(n, np.int64)
    got[pos] = best[root]
    np.testing.assert_array_equal(got.astype(np.uint64), labels_want)


@pytest.mark.parametrize("w,h,make", [
    (256, 256, lambda: synth.cfg1(scale=1_000_000 / (64 * 2**20), seed=91)[0]),
    (448, 512, lambda: synth.cfg4(scale=800_000 / (512 * 2**20), seed=92)[0]),
])
def test_forest_invariants_one_shot(w, h, make):
    hits = make()
    with Clusterer(w, h, 128) as c:
        c.push(hits)
        c.flush()
        parent, pos = c.forest()
    check_forest(hits, parent, pos, oracle.labels(hits, w, h, 128))


def test_forest_general_sort():
    """ToAs more than 2^31 ticks after the first hit (the span stays under
    2^32) leave the tile sort's keys out of range: the general sort orders
    the step, and the forest is read from the buffer its last pass wrote."""
    hits, _ = synth.cfg1(scale=200_000 / (64 * 2**20), seed=93)
    hits = hits.copy()
    hits["toa"][len(hits) // 2:] += np.uint64(2**31 + 2**20)
    assert int(hits["toa"].max()) - int(hits["toa"].min()) < 2**32
    with Clusterer(256, 256, 128) as c:
        c.push(hits)
        c.flush()
        parent, pos = c.forest()
    check_forest(hits, parent, pos, oracle.labels(hits, 256, 256, 128))


def test_forest_streaming_step_and_states():
    hits, t = synth.cfg1(scale=300_000 / (64 * 2**20), seed=94)
    with Clusterer(256, 256, 128) as c:
        with pytest.raises(TpcError) as e:
            c.forest()
        assert e.value.name == "TPC_ERR_STATE"
    with Clusterer(256, 256, 128, max_disorder=t) as c:
        c.push(hits[:150_000])
        carry = c.counts()[2]
        c.push(hits[150_000:])
        parent, pos = c.forest()
        # the step's input: the carried open hits, then the new chunk
        assert len(parent) == carry + len(hits) - 150_000
        assert np.all(parent.astype(np.int64) <= np.arange(len(parent)))
    a, b = Clusterer(256, 256, 128), Clusterer(256, 256, 128)
    try:
        a.push(hits[:1000])
        b.push(hits[1000:2000])
        batch_flush([a, b])
        with pytest.raises(TpcError) as e:
            a.forest()
        assert e.value.name == "TPC_ERR_STATE"
    finally:
        a.close()
        b.close()
