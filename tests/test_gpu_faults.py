"""Failure injection on the host (TPC_OPT_FAIL_ALLOC): every device or pinned
allocation a call sequence makes is made to fail in turn, as an out-of-memory
would.  The call reports TPC_ERR_NOMEM, nothing on the GPU faults (the
allocation is simply not made), the context stays usable, repeating the call
succeeds, and the results equal the oracle's.  The step before a failed step
leaves no readable result behind (its workspace may have been freed)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2412_11809_gb300 import Clusterer, TpcError, batch_flush  # noqa: E402
from paper_2412_11809_gb300.binding import OPT_MAX_DISORDER  # noqa: E402

MAX_SITES = 80


def drive(make, ops, nth):
    """A fresh context, its nth allocation from now failing; an op reporting
    TPC_ERR_NOMEM is repeated once.  Returns (what the ops collected, fired)."""
    got = []
    fired = False
    with make() as c:
        c.inject_alloc_failure(nth)
        for op in ops:
            try:
                r = op(c)
            except TpcError as e:
                assert e.name == "TPC_ERR_NOMEM", e
                assert not fired, "the injected failure fires once"
                fired = True
                r = op(c)
            if r is not None:
                got.append(r)
    return got, fired


def every_site(make, ops, check):
    fired_any = 0
    for nth in range(1, MAX_SITES + 1):
        got, fired = drive(make, ops, nth)
        check(got)
        if not fired:
            break
        fired_any += 1
    else:
        pytest.fail("more allocation sites than expected")
    assert fired_any >= 3, fired_any
    return fired_any


def collect(c):
    lab, idx = c.labels(with_indices=True)
    return idx, lab, c.features()


def check_stream(hits, w=256, h=256, dt=128):
    want = oracle.labels(hits, w, h, dt)
    ref = oracle.features(hits, want)

    def check(got):
        idx = np.concatenate([g[0] for g in got]).astype(np.int64)
        lab = np.concatenate([g[1] for g in got])
        rec = np.concatenate([g[2] for g in got])
        assert len(idx) == len(hits)
        out = np.empty(len(hits), np.uint64)
        out[idx] = lab
        np.testing.assert_array_equal(out, want)
        rec = rec[np.argsort(rec["label"], kind="stable")]
        for k in ("label", "size", "sum_tot", "first_toa"):
            np.testing.assert_array_equal(rec[k], ref[k])
        np.testing.assert_allclose(rec["cx"], ref["cx"], rtol=1e-5)
    return check


@pytest.fixture(scope="module")
def stream():
    hits, t = synth.cfg1(scale=60_000 / (64 * 2**20), seed=81)
    return hits, t


def test_one_shot_host_pushes(stream):
    hits, _ = stream
    a, b = hits[:25_000], hits[25_000:]
    ops = [lambda c: c.push(a), lambda c: c.push(b), lambda c: c.flush(), collect]
    n = every_site(lambda: Clusterer(256, 256, 128), ops, check_stream(hits))
    assert n >= 20       # staging, pending buffer, workspace arrays, outputs


@pytest.fixture(scope="module")
def big():
    """Larger than the workspace's headroom (2^20 positions) above a small
    first step, so that a second step must grow the workspace."""
    hits, t = synth.cfg1(scale=1_300_000 / (64 * 2**20), seed=82)
    return hits, t


def test_one_shot_device_push_and_growth(big):
    """A first small step, then a larger one whose workspace growth may fail:
    the graph captured on the freed arrays must not be replayed."""
    hits, _ = big
    d_small = torch.from_numpy(hits[:3000].view(np.uint8).reshape(-1, 16)).cuda()
    d_all = torch.from_numpy(hits.view(np.uint8).reshape(-1, 16)).cuda()
    small_want = oracle.labels(hits[:3000], 256, 256, 128)
    want = oracle.labels(hits, 256, 256, 128)

    def check_small(c):
        np.testing.assert_array_equal(c.labels(), small_want)

    def shifted(got):
        idx, lab, _ = got[0]
        np.testing.assert_array_equal(idx.astype(np.int64) - 3000, np.arange(len(hits)))
        np.testing.assert_array_equal(lab - 3000, want)

    ops = [lambda c: c.push(d_small), lambda c: c.flush(), check_small,
           lambda c: c.push(d_all), lambda c: c.flush(), collect]
    every_site(lambda: Clusterer(256, 256, 128), ops, shifted)


def test_failed_step_drops_previous_result(stream):
    hits, _ = stream
    with Clusterer(256, 256, 128) as c:
        c.push(hits[:1000])
        c.flush()
        assert len(c.labels()) == 1000
        c.push(hits)                          # needs larger output buffers
        c.inject_alloc_failure(1)
        with pytest.raises(TpcError) as e:
            c.flush()
        assert e.value.name == "TPC_ERR_NOMEM"
        assert len(c.labels()) == 0 and c.counts() == (0, 0, 0)
        c.flush()                             # the pending hits are still there
        lab = c.labels()
        np.testing.assert_array_equal(lab - 1000, oracle.labels(hits, 256, 256, 128))


def test_streaming(stream):
    hits, t = stream
    chunks = np.array_split(hits, 5)
    ops = [lambda c: c.set_option(OPT_MAX_DISORDER, t)]
    for ch in chunks:
        ops += [lambda c, ch=ch: c.push(ch), collect]
    ops += [lambda c: c.flush(), collect]
    n = every_site(lambda: Clusterer(256, 256, 128), ops, check_stream(hits))
    assert n >= 25       # stream state, carry buffers, workspace, outputs, staging


def test_streaming_smaller_chunk_after_failed_growth(big):
    """A failed push is not consumed.  Pushing a smaller chunk instead needs a
    workspace the size of the first step's, the size the graph was captured
    at: after a failed growth it must be captured afresh, never replayed on
    the freed arrays."""
    hits, t = big
    check = check_stream(hits)
    fired_at = []
    for nth in range(1, 16):
        got = []
        with Clusterer(256, 256, 128, max_disorder=t) as c:
            c.push(hits[:4000])
            got.append(collect(c))
            c.inject_alloc_failure(nth)
            try:
                c.push(hits[4000:])           # grows carry buffers, workspace, outputs
                got.append(collect(c))
                fired = False
            except TpcError as e:
                assert e.name == "TPC_ERR_NOMEM"
                fired = True
                c.push(hits[4000:4096])       # a smaller chunk instead
                got.append(collect(c))
                c.push(hits[4096:])
                got.append(collect(c))
            c.flush()
            got.append(collect(c))
        check(got)
        if not fired:
            break
        fired_at.append(nth)
    assert len(fired_at) >= 5, fired_at      # carry buffers (4), then the workspace


@pytest.mark.parametrize("variant", ["static", "global"])
def test_variants(stream, variant):
    hits, _ = stream
    want = oracle.labels(hits, 256, 256, 128, variant)

    def check(got):
        np.testing.assert_array_equal(got[0], want)

    ops = [lambda c: c.push(hits), lambda c: c.flush(), lambda c: c.labels()]
    every_site(lambda: Clusterer(256, 256, 128, variant=variant), ops, check)


def test_batch_with_failing_lead_and_member(stream):
    hits, _ = stream
    parts = np.array_split(hits, 3)
    wants = [oracle.labels(p, 256, 256, 128) for p in parts]
    for victim in (0, 2):
        for nth in range(1, MAX_SITES + 1):
            ctxs = [Clusterer(256, 256, 128) for _ in parts]
            try:
                for c, p in zip(ctxs, parts):
                    c.push(p)
                ctxs[victim].inject_alloc_failure(nth)
                fired = False
                try:
                    batch_flush(ctxs)
                except TpcError as e:
                    assert e.name == "TPC_ERR_NOMEM"
                    fired = True
                    batch_flush(ctxs)
                for c, want in zip(ctxs, wants):
                    np.testing.assert_array_equal(c.labels(), want)
            finally:
                for c in ctxs:
                    c.close()
            if not fired:
                break
        assert nth > 1


def test_restore_with_failures(stream):
    hits, t = stream
    with Clusterer(256, 256, 128, max_disorder=t) as a:
        first = collect_push(a, hits[:30_000])
        snap = a.snapshot()
    for nth in range(1, MAX_SITES + 1):
        with Clusterer(256, 256, 128) as b:
            b.inject_alloc_failure(nth)
            fired = False
            try:
                b.restore(snap)
            except TpcError as e:
                assert e.name == "TPC_ERR_NOMEM"
                fired = True
                b.restore(snap)
            b.inject_alloc_failure(0)
            got = [first, collect_push(b, hits[30_000:])]
            b.flush()
            got.append(collect(b))
        check_stream(hits)(got)
        if not fired:
            break
    assert nth > 2


def collect_push(c, chunk):
    c.push(chunk)
    return collect(c)


def test_option_failure_leaves_context_one_shot(stream):
    """The stream state is allocated before the option is recorded: a failed
    TPC_OPT_MAX_DISORDER leaves a plain one-shot context."""
    hits, t = stream
    with Clusterer(256, 256, 128) as c:
        c.inject_alloc_failure(1)
        with pytest.raises(TpcError) as e:
            c.set_option(OPT_MAX_DISORDER, t)
        assert e.value.name == "TPC_ERR_NOMEM"
        c.push(hits)
        assert c.counts()[0] == 0             # buffered, not streamed
        c.flush()
        np.testing.assert_array_equal(c.labels(), oracle.labels(hits, 256, 256, 128))
