"""The serving loop (tpc_server_*): detector streams under one device-memory
budget, chunks admitted as memory frees up, their work overlapping on the GPU.
Each stream's results must be the same through the server (in the mix, with
queueing forced by a tight budget), through its own streaming context alone,
and as the one-shot oracle's on the whole stream (open clusters carried on
the device must not change any cluster: Section 3.3, Algorithm 2)."""
import numpy as np
import pytest

import synth
from gpu_helpers import assert_features_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2412_11809_gb300 import Clusterer, Server  # noqa: E402
from test_gpu_serving import check_stream_result, collect_stream  # noqa: E402


def _run_server(server, streams, ids):
    """Submit every chunk of every stream at once (interleaved), then the
    ends of the streams; gather per stream (indices, labels, records)."""
    out = {k: ([], [], []) for k in ids}
    tag = 0
    order = []
    for j in range(max(len(s[1]) for s in streams)):
        for k, (hits, sizes, _) in zip(ids, streams):
            if j < len(sizes):
                start = int(np.sum(sizes[:j]))
                order.append((k, hits[start:start + sizes[j]]))
    for k, chunk in order:
        server.submit(k, chunk, tag)
        tag += 1
    for k in ids:
        server.submit(k, None, tag, cap=1 << 20, end=True)
        tag += 1
    for _ in range(tag):
        r, lab, idx, rec = server.wait(timeout_s=120)
        assert r.status == 0, f"chunk {r.tag} of stream {r.stream}: status {r.status}"
        out[r.stream][0].append(idx.copy())
        out[r.stream][1].append(lab.copy())
        out[r.stream][2].append(rec.copy())
    return {k: tuple(np.concatenate(v) for v in vals) for k, vals in out.items()}


def test_server_tight_budget_queues_and_matches_alone_and_oracle():
    """Two streams whose first chunks (1 Mi hits each) cannot run together
    under the budget: a 1 Mi-hit first chunk holds about 280 B per hit while
    it runs (work arrays, outputs, the stream's carry and chunk buffers), and
    about half of that stays held by the idle stream (its carry and chunk
    buffers).  The second stream's first chunk is submitted microseconds
    after the first one, which takes milliseconds, so it must wait at the
    head of the queue; once the first finishes, the idle stream's work
    arrays are released and it fits.  The later chunks (64k-128k hits) run
    side by side."""
    rng = np.random.default_rng(77)
    streams = []
    for hits, _, t in synth.cfg3(hits_per_stream=3_000_000, n_streams=2, seed=77):
        sizes = [2**20]
        while sum(sizes) < len(hits):
            sizes.append(min(int(rng.integers(65536, 131073)), len(hits) - sum(sizes)))
        streams.append((hits, np.array(sizes), t))
    budget = 512 << 20
    with Server(budget) as srv:
        ids = [srv.add_stream(256, 256, 128, t) for _, _, t in streams]
        got = _run_server(srv, streams, ids)
        st = srv.stats()
    assert st["waits"] > 0, f"the budget should have made chunks wait: {st}"
    assert st["releases"] > 0, st
    assert st["peak"] <= budget
    assert st["completed"] == st["submitted"] and st["failed"] == 0 and st["rejected"] == 0, st
    for k, (hits, sizes, t) in zip(ids, streams):
        idx, lab, rec = got[k]
        check_stream_result(hits, idx, lab, rec)   # against the oracle on the whole stream
        with Clusterer(256, 256, 128, max_disorder=t) as c:   # the same stream alone
            a_idx, a_lab, a_rec = collect_stream(c, hits, sizes)
        np.testing.assert_array_equal(lab[np.argsort(idx)], a_lab[np.argsort(a_idx)])
        assert_features_equal(np.sort(rec, order="label"), np.sort(a_rec, order="label"))


def test_server_roomy_budget_no_waits():
    streams = synth.cfg3(hits_per_stream=300_000, n_streams=3, seed=78, chunk_lo=65536,
                         chunk_hi=131072)
    with Server(4 << 30) as srv:
        ids = [srv.add_stream(256, 256, 128, t) for _, _, t in streams]
        got = _run_server(srv, streams, ids)
        st = srv.stats()
    assert st["waits"] == 0 and st["releases"] == 0
    for k, (hits, _, _) in zip(ids, streams):
        check_stream_result(hits, *got[k])


def test_server_rejects_a_chunk_that_can_never_fit():
    hits, t = synth.cfg1(scale=1 / 16, seed=79)          # 4 Mi hits: far above the budget
    with Server(64 << 20) as srv:
        k = srv.add_stream(256, 256, 128, t)
        srv.submit(k, hits, 1)
        r, _, _, _ = srv.wait(timeout_s=60)
        assert r.tag == 1 and r.status == -4          # TPC_ERR_BUSY
        small = hits[:50_000]                           # the stream stays usable
        srv.submit(k, small, 2)
        srv.submit(k, None, 3, cap=1 << 20, end=True)
        idx, lab, rec = [], [], []
        for _ in range(2):
            r, l_, i_, c_ = srv.wait(timeout_s=60)
            assert r.status == 0
            idx.append(i_.copy()); lab.append(l_.copy()); rec.append(c_.copy())
        st = srv.stats()
    assert st["rejected"] == 1
    check_stream_result(small, np.concatenate(idx), np.concatenate(lab), np.concatenate(rec))
