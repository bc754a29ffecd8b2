"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the oracle element by element."""
import numpy as np

import oracle
from paper_2412_11809_gb300 import Clusterer

CENTROID_RTOL = 1e-5   # fp32 centroid vs the fp64 oracle


def run_gpu(hits, width, height, dt, variant="local", device=True, pushes=1, **kw):
    import torch
    with Clusterer(width, height, dt, variant, **kw) as c:
        parts = np.array_split(hits, pushes) if pushes > 1 else [hits]
        for p in parts:
            if device:
                c.push(torch.from_numpy(np.ascontiguousarray(p).view(np.uint8).reshape(-1, 16)).cuda())
            else:
                c.push(p)
        c.flush()
        lab = c.labels()
        feats = c.features()
    return lab, feats


def assert_features_equal(got, want):
    assert len(got) == len(want), (len(got), len(want))
    for k in ("label", "size", "sum_tot", "first_toa"):
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    for k in ("cx", "cy"):
        w = want[k]
        g = got[k].astype(np.float64)
        nan = np.isnan(w)
        np.testing.assert_array_equal(np.isnan(g), nan, err_msg=k)
        np.testing.assert_allclose(g[~nan], w[~nan], rtol=CENTROID_RTOL, atol=0, err_msg=k)


def check_against_oracle(hits, width, height, dt, variant="local", **kw):
    lab, feats = run_gpu(hits, width, height, dt, variant, **kw)
    want = oracle.labels(hits, width, height, dt, variant)
    if not np.array_equal(lab, want):
        bad = np.flatnonzero(lab != want)
        raise AssertionError(f"{len(bad)} of {len(want)} labels differ; first at {bad[:5]}: "
                             f"got {lab[bad[:5]]} want {want[bad[:5]]}")
    assert_features_equal(feats, oracle.features(hits, want))
    return lab, feats


def sampled_cluster_check(hits, labels, width, height, dt, n_samples, rng):
    """Exact check of sampled clusters of a large run: the oracle clusters a
    time window around each sampled cluster, widened until no hit within dt
    of the window's edge belongs to the component; the component must equal
    the GPU cluster as an index set.  Valid for variant (a), whose components
    only depend on hits within dt along the way."""
    order = np.argsort(hits["toa"], kind="stable")
    toa_sorted = hits["toa"][order]
    picks = rng.choice(len(hits), size=n_samples, replace=False)
    by_label = {}
    for i in picks:
        lab = int(labels[i])
        if lab in by_label:
            continue
        members = np.flatnonzero(labels == lab) if lab not in by_label else by_label[lab]
        by_label[lab] = members
        lo = int(hits["toa"][members].min())
        hi = int(hits["toa"][members].max())
        while True:
            a = np.searchsorted(toa_sorted, np.uint64(max(lo - 2 * dt, 0)), side="left")
            b = np.searchsorted(toa_sorted, np.uint64(hi + 2 * dt), side="right")
            idx = np.sort(order[a:b])
            sub = hits[idx]
            sl = oracle.labels(sub, width, height, dt)
            pos = int(np.searchsorted(idx, i))
            comp = idx[sl == sl[pos]]
            clo, chi = int(hits["toa"][comp].min()), int(hits["toa"][comp].max())
            if clo - dt > lo - 2 * dt and chi + dt < hi + 2 * dt:
                break
            lo, hi = min(lo, clo), max(hi, chi)
        assert np.array_equal(np.sort(comp), members), f"cluster of hit {i} differs"
        assert int(members.min()) == lab
    return len(by_label)
