"""The library's hit buffer filling (Algorithm 2, host code behind the C ABI,
no GPU needed) against the oracle's: the same buffers, hit for hit, the same
arrival numbers and the same cuts, whatever the chunking of the stream."""
import numpy as np
import pytest

import oracle
import synth

from paper_2412_11809_gb300 import Filler, TpcError


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_2412_11809_gb300 import build
    build.build()


def run_filler(hits, params, chunks):
    got = []
    with Filler(*params) as f:
        start = 0
        for c in chunks:
            f.store(hits[start:start + c])
            start += c
            while (b := f.take()) is not None:
                got.append(b)
        f.finish()
        f.finish()                       # idempotent
        while (b := f.take()) is not None:
            got.append(b)
        with pytest.raises(TpcError) as e:
            f.store(hits[:1])
        assert e.value.name == "TPC_ERR_STATE"
    return got


def expect_from_oracle(hits, params):
    buf, cut = oracle.fill_buffers(hits, *params)
    return [(np.nonzero(buf == k)[0], cut[k]) for k in range(len(cut))]


def assert_same(hits, got, want):
    assert len(got) == len(want)
    for (h, idx, cut), (widx, wcut) in zip(got, want):
        np.testing.assert_array_equal(idx, widx)
        np.testing.assert_array_equal(h, hits[widx])
        assert cut == wcut


def test_worked_example_fixture():
    from test_oracle_filling import FIXTURE, load_fixture
    hits, params, buf, cut = load_fixture(FIXTURE)
    got = run_filler(hits, params, [len(hits)])
    assert_same(hits, got, [(np.nonzero(buf == k)[0], cut[k]) for k in range(len(cut))])
    got1 = run_filler(hits, params, [1] * len(hits))       # one hit per call
    assert_same(hits, got1, [(np.nonzero(buf == k)[0], cut[k]) for k in range(len(cut))])


@pytest.mark.parametrize("params", [(40_000, 12_000, None, 200), (3000, 100, None, 0),
                                    (800, 700, None, 20), (5, 2, 3, 2), (1, 0, None, 0),
                                    (10**9, 1, None, 100)])
def test_equals_oracle_on_t_ordered_stream(params):
    hits, t = synth.cfg1(scale=250_000 / (64 * 2**20), seed=21)
    if params[0] < 100:
        hits = hits[:5000]               # tiny buffers: one Python call per buffer
    params = tuple(t if v is None else v for v in params)
    want = expect_from_oracle(hits, params)
    rng = np.random.default_rng(5)
    chunks = []
    while sum(chunks) < len(hits):
        chunks.append(int(min(len(hits) - sum(chunks), rng.integers(1, 30_000))))
    assert_same(hits, run_filler(hits, params, chunks), want)
    assert_same(hits, run_filler(hits, params, [len(hits)]), want)


def test_equals_oracle_on_unordered_input():
    """Any input, not only t-ordered streams: the procedure is the same."""
    rng = np.random.default_rng(9)
    n = 20_000
    hits = oracle.make_hits(rng.integers(0, 256, n), rng.integers(0, 256, n),
                            rng.integers(0, 10**6, n, dtype=np.uint64))
    for params in [(1000, 300, 5000, 100), (64, 63, 0, 0), (2000, 0, 10**5, 10**4)]:
        want = expect_from_oracle(hits, params)
        assert_same(hits, run_filler(hits, params, [777] * (n // 777) + [n % 777]), want)


def test_saturating_times():
    top = 2**64 - 10
    hits = oracle.make_hits([0] * 6, [0] * 6,
                            np.array([top - 5, top - 6, top - 2, top, 3, top - 1], dtype=np.uint64))
    params = (4, 2, 2**64 - 1, 2**63)
    assert_same(hits, run_filler(hits, params, [6]), expect_from_oracle(hits, params))


def test_arguments():
    for b, b_t in [(0, 0), (4, 4), (4, 9)]:
        with pytest.raises(TpcError):
            Filler(b, b_t, 10, 1)
    with Filler(10, 2, 5, 1) as f:
        assert f.take() is None and f.ready() == (0, 0)
        f.store(np.zeros(0, dtype=oracle.HIT_DTYPE))
        f.finish()
        assert f.take() is None
