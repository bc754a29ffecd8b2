"""Pins for the CPU oracle against what the paper and the mathematics fix.

* hand-derived fixtures (``tests/golden``) for the three temporal conditions
  of Section 2 (iii) and the cluster features;
* O(n^2) brute force + scipy connected components for variant (a);
* an independently written sweep for variants (b) and (c);
* the large-dt limit where all variants reduce to textbook 8-connected CCL of
  the occupied pixels (Section 2: "for large values of dt ... identical");
* refinement (c) <= (a) <= (b), dt monotonicity, input-order independence;
* the defining invariants on generated workloads.
"""
import numpy as np
import pytest

import oracle
import synth
from bruteforce import (local_bruteforce, pixel_ccl, random_hits, refines,
                        sweep_bruteforce)
from golden_cases import all_cases

VARIANTS = ("local", "global", "static")


@pytest.mark.parametrize("case", all_cases(), ids=lambda c: c["name"])
def test_golden_labels(case):
    for v, want in case["expect"].items():
        got = oracle.labels(case["hits"], case["width"], case["height"], case["dt"], v)
        np.testing.assert_array_equal(got, want, err_msg=f"{case['name']} variant {v}")


@pytest.mark.parametrize("case", [c for c in all_cases() if c["features"]],
                         ids=lambda c: c["name"])
def test_golden_features(case):
    lab = oracle.labels(case["hits"], case["width"], case["height"], case["dt"])
    f = oracle.features(case["hits"], lab)
    assert len(f) == len(case["features"])
    for rec, (label, size, sum_tot, first, cx, cy) in zip(f, case["features"]):
        assert (rec["label"], rec["size"], rec["sum_tot"], rec["first_toa"]) == \
            (label, size, sum_tot, first)
        assert rec["cx"] == pytest.approx(cx, rel=1e-15)
        assert rec["cy"] == pytest.approx(cy, rel=1e-15)


@pytest.mark.parametrize("seed", range(60))
def test_local_matches_bruteforce(seed):
    rng = np.random.default_rng(seed)
    w = int(rng.integers(1, 12))
    h = int(rng.integers(1, 12))
    n = int(rng.integers(0, 260))
    span = int(rng.integers(0, 400))
    dt = int(rng.integers(0, 60))
    hits = random_hits(rng, n, w, h, span)
    np.testing.assert_array_equal(oracle.labels(hits, w, h, dt, "local"),
                                  local_bruteforce(hits, dt))


@pytest.mark.parametrize("variant", ["global", "static"])
@pytest.mark.parametrize("seed", range(40))
def test_sweep_matches_independent_sweep(seed, variant):
    rng = np.random.default_rng(1000 + seed)
    w = int(rng.integers(1, 10))
    h = int(rng.integers(1, 10))
    n = int(rng.integers(0, 120))
    span = int(rng.integers(0, 300))
    dt = int(rng.integers(0, 50))
    hits = random_hits(rng, n, w, h, span)
    np.testing.assert_array_equal(oracle.labels(hits, w, h, dt, variant),
                                  sweep_bruteforce(hits, dt, variant))


@pytest.mark.parametrize("seed", range(10))
def test_large_dt_limit_is_pixel_ccl(seed):
    """dt >= ToA span: every temporal condition holds, so all three variants
    are plain 8-connected labelling of the occupied pixels."""
    rng = np.random.default_rng(2000 + seed)
    w, h = int(rng.integers(2, 40)), int(rng.integers(2, 40))
    hits = random_hits(rng, int(rng.integers(1, 400)), w, h, 1000)
    want = pixel_ccl(hits, w, h)
    for v in VARIANTS:
        np.testing.assert_array_equal(oracle.labels(hits, w, h, 1000, v), want)


def test_refinement_and_monotonicity():
    hits, _ = synth.cfg1(scale=1 / 512, seed=7)
    a = oracle.labels(hits, 256, 256, 128, "local")
    b = oracle.labels(hits, 256, 256, 128, "global")
    c = oracle.labels(hits, 256, 256, 128, "static")
    assert refines(c, a) and refines(a, b)
    a_wide = oracle.labels(hits, 256, 256, 384, "local")
    assert refines(a, a_wide)
    # the workload must actually exercise the differences
    assert len(np.unique(c)) > len(np.unique(a)) > len(np.unique(b))


@pytest.mark.parametrize("variant", VARIANTS)
def test_input_order_independence(variant):
    hits, _ = synth.cfg1(scale=1 / 1024, seed=11)
    base = oracle.labels(hits, 256, 256, 128, variant)
    rng = np.random.default_rng(5)
    perm = rng.permutation(len(hits))
    got = oracle.labels(hits[perm], 256, 256, 128, variant)
    # cluster of original hit perm[k] is got[k] (a position in the permuted input);
    # map it back to the original index and compare partitions
    members = {}
    for k in range(len(perm)):
        members.setdefault(int(got[k]), []).append(int(perm[k]))
    relabel = np.empty(len(hits), dtype=np.uint64)
    for m in members.values():
        relabel[m] = min(m)
    np.testing.assert_array_equal(relabel, base)


def test_equal_toa_ties_order_free():
    """Many hits share a ToA; any order among them gives the same partition."""
    rng = np.random.default_rng(3)
    hits = random_hits(rng, 300, 10, 10, 0)
    hits["toa"] = rng.integers(0, 6, len(hits)).astype(np.uint64) * 7
    for v in VARIANTS:
        base = oracle.labels(hits, 10, 10, 7, v)
        perm = rng.permutation(len(hits))
        got = oracle.labels(hits[perm], 10, 10, 7, v)
        inv = np.argsort(perm)
        back = got[inv]              # label (in permuted positions) of each original hit
        remap = perm[back.astype(np.int64)]
        groups = {}
        for i, g in enumerate(remap):
            groups.setdefault(int(g), []).append(i)
        relabel = np.empty(len(hits), dtype=np.uint64)
        for m in groups.values():
            relabel[m] = min(m)
        np.testing.assert_array_equal(relabel, base, err_msg=v)


def _clusters(lab):
    order = np.argsort(lab, kind="stable")
    bounds = np.flatnonzero(np.diff(lab[order])) + 1
    return np.split(order, bounds)


def _spatially_connected(xs, ys):
    pts = list(zip(xs.tolist(), ys.tolist()))
    seen = {0}
    stack = [0]
    while stack:
        i = stack.pop()
        for j in range(len(pts)):
            if j not in seen and abs(pts[i][0] - pts[j][0]) <= 1 and abs(pts[i][1] - pts[j][1]) <= 1:
                seen.add(j)
                stack.append(j)
    return len(seen) == len(pts)


def test_definition_invariants_on_workload():
    hits, _ = synth.cfg1(scale=1 / 1024, seed=13)
    dt = 128
    for v in VARIANTS:
        lab = oracle.labels(hits, 256, 256, dt, v)
        # canonical: label is the smallest member index and a fixed point
        assert np.all(lab <= np.arange(len(hits)))
        assert np.all(lab[lab.astype(np.int64)] == lab)
        for members in _clusters(lab):
            assert lab[members[0]] == members.min()
            if len(members) == 1:
                continue
            assert _spatially_connected(hits["x"][members], hits["y"][members])
            t = np.sort(hits["toa"][members].astype(np.int64))
            if v == "global":
                assert np.all(np.diff(t) <= dt)
            if v == "static":
                assert t[-1] - t[0] <= dt
    # (a) maximality: no edge of the hit graph crosses two clusters
    lab = oracle.labels(hits, 256, 256, dt, "local")
    order = np.argsort(hits["toa"], kind="stable")
    t = hits["toa"][order].astype(np.int64)
    x = hits["x"][order].astype(np.int64)
    y = hits["y"][order].astype(np.int64)
    lo = 0
    for k in range(len(order)):
        while t[k] - t[lo] > dt:
            lo += 1
        near = slice(lo, k)
        adj = (np.abs(x[near] - x[k]) <= 1) & (np.abs(y[near] - y[k]) <= 1)
        assert np.all(lab[order[near][adj]] == lab[order[k]])


def test_features_invariants():
    hits, _ = synth.cfg1(scale=1 / 256, seed=17)
    lab = oracle.labels(hits, 256, 256, 128)
    f = oracle.features(hits, lab)
    assert np.all(np.diff(f["label"].astype(np.int64)) > 0)
    assert set(f["label"].tolist()) == set(np.unique(lab).tolist())
    assert f["size"].sum() == len(hits)
    assert f["sum_tot"].sum() == hits["tot"].astype(np.int64).sum()
    first = np.full(len(hits), np.iinfo(np.uint64).max, dtype=np.uint64)
    np.minimum.at(first, lab.astype(np.int64), hits["toa"])
    np.testing.assert_array_equal(f["first_toa"], first[f["label"].astype(np.int64)])
    xmin = np.full(len(hits), 1 << 20); xmax = np.zeros(len(hits), np.int64)
    np.minimum.at(xmin, lab.astype(np.int64), hits["x"].astype(np.int64))
    np.maximum.at(xmax, lab.astype(np.int64), hits["x"].astype(np.int64))
    li = f["label"].astype(np.int64)
    assert np.all(f["cx"] >= xmin[li]) and np.all(f["cx"] <= xmax[li])
    single = f["size"] == 1
    np.testing.assert_array_equal(f["cx"][single], hits["x"][li[single]])
    np.testing.assert_array_equal(f["cy"][single], hits["y"][li[single]])


def test_edge_inputs():
    empty = np.zeros(0, dtype=oracle.HIT_DTYPE)
    for v in VARIANTS:
        assert len(oracle.labels(empty, 4, 4, 10, v)) == 0
    assert len(oracle.features(empty, np.zeros(0, np.uint64))) == 0
    one = oracle.make_hits([3], [2], [5])
    for v in VARIANTS:
        np.testing.assert_array_equal(oracle.labels(one, 4, 3, 0, v), [0])
    # all hits on one pixel, one tick apart: one cluster iff dt >= 1
    pile = oracle.make_hits(np.zeros(50, int), np.zeros(50, int), np.arange(50)[::-1])
    for v in ("local", "global"):
        assert len(np.unique(oracle.labels(pile, 1, 1, 1, v))) == 1
        assert len(np.unique(oracle.labels(pile, 1, 1, 0, v))) == 50
    # (c) with dt = 10 on a 1-tick chain: windows of 11 hits from each cluster's first
    assert len(np.unique(oracle.labels(pile, 1, 1, 10, "static"))) == 5


def test_toa_near_wraparound():
    top = np.iinfo(np.uint64).max
    hits = oracle.make_hits([0, 1, 2], [0, 0, 0],
                            np.array([top, top - 5, top - 16], dtype=np.uint64))
    for v in VARIANTS:
        lab = oracle.labels(hits, 3, 1, 5, v)
        np.testing.assert_array_equal(lab, [0, 0, 2])


def test_out_of_range_rejected():
    bad = oracle.make_hits([4], [0], [0])
    with pytest.raises(ValueError):
        oracle.labels(bad, 4, 4, 10)


def test_concurrent_calls_agree_with_sequential():
    """The oracle is called from several threads at once by the full-size
    tests (the C library releases the GIL): each thread's result must equal
    the same call made alone."""
    import threading
    streams = [synth.cfg1(scale=1 / 512, seed=900 + k)[0] for k in range(4)]
    want = [oracle.labels(h, 256, 256, 128, v) for h, v in zip(streams, ("local", "global", "static", "local"))]
    got = [None] * 4

    def run(k, v):
        got[k] = oracle.labels(streams[k], 256, 256, 128, v)

    threads = [threading.Thread(target=run, args=(k, v))
               for k, v in enumerate(("local", "global", "static", "local"))]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    for g, w in zip(got, want):
        np.testing.assert_array_equal(g, w)
