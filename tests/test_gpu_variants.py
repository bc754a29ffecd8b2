"""Variants (iii)(b) and (iii)(c) of the cluster definition (paper Section 2)
on the device, against the oracle's time sweep (Algorithm 1 reading):
labels bit-exact, integer features exact, centroids within 1e-5 relative.
Also every hand-derived golden fixture through the CUDA path."""
import numpy as np
import pytest

import oracle
import synth
from bruteforce import random_hits
from golden_cases import all_cases
from gpu_helpers import check_against_oracle, run_gpu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("case", all_cases(), ids=lambda c: c["name"])
def test_golden_all_variants(case):
    for v, want in case["expect"].items():
        lab, _ = run_gpu(case["hits"], case["width"], case["height"], case["dt"], v)
        np.testing.assert_array_equal(lab, want, err_msg=f"{case['name']} {v}")


@pytest.mark.parametrize("variant", ["global", "static"])
def test_cfg0_scaled(variant):
    hits, _ = synth.cfg0(scale=0.25, seed=21)
    check_against_oracle(hits, 256, 256, 128, variant)


@pytest.mark.parametrize("variant", ["global", "static"])
@pytest.mark.parametrize("dt", [128, 384])
def test_cfg1_scaled(variant, dt):
    hits, _ = synth.cfg1(scale=1 / 64, seed=22)
    check_against_oracle(hits, 256, 256, dt, variant)


@pytest.mark.parametrize("variant", ["global", "static"])
def test_cfg4_timepix4_scaled(variant):
    hits, _ = synth.cfg4(scale=1 / 512, seed=23)
    check_against_oracle(hits, 448, 512, 128, variant)


@pytest.mark.parametrize("variant", ["global", "static"])
@pytest.mark.parametrize("seed", range(6))
def test_random_dense(variant, seed):
    rng = np.random.default_rng(300 + seed)
    w, h = int(rng.integers(1, 12)), int(rng.integers(1, 12))
    n = int(rng.integers(2000, 12000))
    hits = random_hits(rng, n, w, h, int(rng.integers(0, 3 * n)))
    check_against_oracle(hits, w, h, int(rng.integers(0, 40)), variant)


@pytest.mark.parametrize("dt", [30, 400])
def test_global_long_timelines_busy_neighbour(dt):
    """(b) with pixel timelines of thousands of hits, so that warps take
    whole 32-hit chunks of one pixel and carry their neighbour cursors from
    chunk to chunk, next to a pixel firing 20 times as often: 32 hits of a
    quiet pixel then span hundreds of the busy one's, past the 64-entry
    window each lane searches first."""
    rng = np.random.default_rng(77 + dt)
    w = h = 6
    n = 120_000
    weights = np.ones(w * h)
    weights[14] = 20.0
    px = rng.choice(w * h, size=n, p=weights / weights.sum())
    t = np.sort(rng.integers(0, n * 40, size=n))
    hits = oracle.make_hits(px % w, px // w, t)
    check_against_oracle(hits, w, h, dt, "global")


@pytest.mark.parametrize("variant", ["global", "static"])
def test_edge_cases(variant):
    one = oracle.make_hits([3], [2], [5])
    check_against_oracle(one, 4, 3, 0, variant)
    pile = oracle.make_hits(np.zeros(5000, int), np.zeros(5000, int), np.arange(5000)[::-1] * 2)
    check_against_oracle(pile, 1, 1, 3, variant)
    check_against_oracle(pile, 1, 1, 1, variant)
    rng = np.random.default_rng(9)
    same = random_hits(rng, 8000, 60, 40, 0)
    check_against_oracle(same, 60, 40, 0, variant)


def test_refinement_on_device():
    hits, _ = synth.cfg1(scale=1 / 128, seed=24)
    a, _ = run_gpu(hits, 256, 256, 128, "local")
    b, _ = run_gpu(hits, 256, 256, 128, "global")
    c, _ = run_gpu(hits, 256, 256, 128, "static")
    ai, bi, ci = (x.astype(np.int64) for x in (a, b, c))
    assert np.all(a == a[ci])      # (c) refines (a)
    assert np.all(b == b[ai])      # (a) refines (b)


def _gpu_stats(hits, w, h, dt, variant):
    from paper_2412_11809_gb300 import Clusterer
    with Clusterer(w, h, dt, variant) as c:
        c.push(hits)
        c.flush()
        lab = c.labels()
        st = c.variant_stats()
    np.testing.assert_array_equal(lab, oracle.labels(hits, w, h, dt, variant))
    return st


def test_device_paths_are_reached():
    """The paths the large workloads take, each against the oracle: (c)
    components longer than the shared-memory staging swept through the
    sliding window, and swept again from global memory when more hits than
    the window holds lie within dt; (b) several rounds over the open-edge
    list, with an exact recomputation of the groups' last ToA at the end, and
    full passes when that list overflows."""
    hits, _ = synth.cfg4(scale=1 / 128, seed=25)          # 4 Mi hits at 2.5 Ghits/s density
    st = _gpu_stats(hits, 448, 512, 128, "static")
    assert st["windowed"] > 0 and st["window_fallbacks"] == 0, st
    st = _gpu_stats(hits, 448, 512, 128, "global")
    assert st["rounds"] >= 3 and st["exact_checks"] >= 1 and st["first_open_edges"] > 0, st
    rng = np.random.default_rng(31)
    same = random_hits(rng, 9000, 60, 40, 0)               # one ToA: every hit within dt of every other
    st = _gpu_stats(same, 60, 40, 0, "static")            # a 9000-hit component: the CTA sweep, global
    assert st["windowed"] > 0 and st["window_fallbacks"] == st["windowed"] == st["global_sweeps"], st
    big = random_hits(rng, 3000, 60, 40, 0)                # 3000 within dt: the CTA sweep, staged
    st = _gpu_stats(big, 60, 40, 0, "static")
    assert st["window_fallbacks"] > 0 and st["global_sweeps"] == 0, st
    # every pixel of a 30 x 30 sensor fires 20 times at random, far apart in
    # time: almost every hit's 9 latest neighbours lie in other, closed groups,
    # more open edges than the list holds; plus one merge that only (b) makes
    # (h joins L's group through its member M, which h is not adjacent to)
    t = rng.integers(0, 10**7, size=(900, 20))
    px = np.repeat(np.arange(900), 20)
    bg = oracle.make_hits(px % 30, px // 30, t.ravel())
    lmh = oracle.make_hits([10, 11, 9], [10, 11, 10], [20_000_000, 20_000_003, 20_000_005])  # L, M, h
    mix = np.concatenate([bg, lmh.astype(bg.dtype)])
    mix = mix[np.argsort(mix["toa"], kind="stable")]
    st = _gpu_stats(mix, 30, 30, 3, "global")
    assert st["full_rounds"] >= 2 and st["rounds"] >= 2, st   # the open-edge list overflowed
