"""Algorithm 3, steps 1-2 end to end: the host-side hit buffer filling of
Algorithm 2 sends its buffers to a streaming context (tpc_filler_send), and
the clusters equal the oracle's on the stream as it arrived.  The buffers
change the order of hits (a late hit can be sent before an earlier arrival),
so labels are compared as partitions: each cluster's smallest arrival number."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2412_11809_gb300 import Clusterer, Filler  # noqa: E402


def cluster_through_filler(hits, t, params, chunk, dt=128):
    n = len(hits)
    arrival_of_push = []          # arrival number of each pushed hit, push order
    push_idx, push_lab = [], []
    with Clusterer(256, 256, dt, max_disorder=t) as c, Filler(*params) as f:
        def drain():
            while (r := f.send(c)) is not None:
                arrival_of_push.append(r[0])
                lab, idx = c.labels(with_indices=True)
                push_idx.append(idx)
                push_lab.append(lab)
        for s in range(0, n, chunk):
            f.store(hits[s:s + chunk])
            drain()
        f.finish()
        drain()
        c.flush()
        lab, idx = c.labels(with_indices=True)
        push_idx.append(idx)
        push_lab.append(lab)
    arrival = np.concatenate(arrival_of_push).astype(np.int64)
    idx = np.concatenate(push_idx).astype(np.int64)
    lab = np.concatenate(push_lab).astype(np.int64)
    assert len(arrival) == n and len(idx) == n
    np.testing.assert_array_equal(np.sort(arrival), np.arange(n))
    np.testing.assert_array_equal(np.sort(idx), np.arange(n))
    # label of each pushed hit in push numbering -> smallest arrival number
    lab_of_push = np.empty(n, np.int64)
    lab_of_push[idx] = lab
    best = np.full(n, n, np.int64)
    np.minimum.at(best, lab_of_push, arrival)
    got = np.empty(n, np.uint64)
    got[arrival] = best[lab_of_push]
    return got


@pytest.mark.parametrize("params,chunk", [((200_000, 40_000, None, 200), 65_536),
                                          ((30_000, 500, None, 0), 10_000),
                                          ((4_000, 3_000, None, 50), 100_000)])
def test_filler_into_streaming_context_equals_oracle(params, chunk):
    hits, t = synth.cfg1(scale=1_000_000 / (64 * 2**20), seed=31)
    params = tuple(t if v is None else v for v in params)
    got = cluster_through_filler(hits, t, params, chunk)
    np.testing.assert_array_equal(got, oracle.labels(hits, 256, 256, 128))
