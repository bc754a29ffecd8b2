"""The autotuner of the batched step (tpc_tune_batch) and the launch choices
it sets (tpc_tuning): every choice gives labels and records identical to the
oracle's (results never depend on launch choices), the tuner leaves the
batch pending, writes its choice to the cache file and reads it back for a
batch with the same key."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import assert_features_equal

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2412_11809_gb300 import Clusterer, Tuning, batch_flush, tune_batch  # noqa: E402


def _batch(scale, seed):
    dets = synth.cfg2(scale=scale, seed=seed)
    ctxs = [Clusterer(w, h, 128) for w, h, _, _, _ in dets]
    d_hits = [torch.from_numpy(h.view(np.uint8).reshape(-1, 16)).cuda() for _, _, h, _, _ in dets]
    return dets, ctxs, d_hits


def _check(dets, ctxs, base=0):
    """Labels are global stream indices: after `base` earlier hits per
    detector, the oracle's labels shifted by base."""
    for c, (w, h, hits, _, _) in zip(ctxs, dets):
        want = oracle.labels(hits, w, h, 128)
        np.testing.assert_array_equal(c.labels() - np.uint64(base * len(hits)), want)
        rec = c.features()
        rec["label"] -= np.uint64(base * len(hits))
        assert_features_equal(rec, oracle.features(hits, want))


@pytest.mark.parametrize("choice", [
    {"acc_span": 512}, {"acc_span": 2048}, {"general_link": 3}, {"general_link": 2, "order": 1},
    {"ctas_sort": 1, "ctas_link": 1, "ctas_acc": 1, "ctas_out": 1}])
def test_every_launch_choice_matches_oracle(choice):
    dets, ctxs, d_hits = _batch(1 / 128, 21)
    ctxs[0].set_tuning(choice)
    assert {k: ctxs[0].tuning().as_dict()[k] for k in choice} == choice
    for c, d in zip(ctxs, d_hits):
        c.push(d)
    batch_flush(ctxs)
    _check(dets, ctxs)
    with Clusterer(448, 512, 128) as single:   # a single context's steps use its choices too
        single.set_tuning(choice)
        hits = dets[-1][2]
        single.push(hits)
        single.flush()
        np.testing.assert_array_equal(single.labels(), oracle.labels(hits, 448, 512, 128))
    for c in ctxs:
        c.close()


def test_tuner_chooses_caches_and_keeps_results(tmp_path):
    cache = str(tmp_path / "tune.txt")
    dets, ctxs, d_hits = _batch(1 / 32, 22)
    for c, d in zip(ctxs, d_hits):
        c.push(d)
    rep = tune_batch(ctxs, cache)
    assert not rep.from_cache and rep.trials > 10
    assert rep.untuned_ms > 0 and rep.tuned_ms <= rep.untuned_ms
    assert ctxs[0].tuning().as_dict() == rep.chosen.as_dict()
    batch_flush(ctxs)            # the tuned batch: the hits were left pending
    _check(dets, ctxs)
    # the same geometries and size buckets: the cached choice, nothing timed
    for c, d in zip(ctxs, d_hits):
        c.push(d)
    ctxs[0].set_tuning(None)
    rep2 = tune_batch(ctxs, cache)
    assert rep2.from_cache and rep2.trials == 0 and rep2.key == rep.key
    assert rep2.chosen.as_dict() == rep.chosen.as_dict()
    assert ctxs[0].tuning().as_dict() == rep.chosen.as_dict()
    batch_flush(ctxs)
    _check(dets, ctxs, base=1)   # each detector's stream went on after its first batch
    for c in ctxs:
        c.close()


def test_tuner_needs_pending_hits():
    from paper_2412_11809_gb300 import TpcError
    with Clusterer(256, 256, 128) as c:
        with pytest.raises(TpcError):
            tune_batch([c])
    t = Tuning(acc_span=777)
    with Clusterer(256, 256, 128) as c:
        with pytest.raises(TpcError):
            c.set_tuning(t)
