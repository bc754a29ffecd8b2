"""Independent brute-force references used to pin the oracle (tiny inputs only).

None of this shares code with ``oracle/``: the (a) reference is an O(n^2)
adjacency matrix handed to scipy's connected-components routine, and the
(b)/(c) reference is a separately written sweep that keeps clusters as plain
Python sets and scans every cluster for every hit.
"""
import numpy as np
from scipy import ndimage
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import connected_components


def canonical(comp: np.ndarray) -> np.ndarray:
    """Relabel a component-id array so each hit carries the smallest index of its component."""
    comp = np.asarray(comp)
    n = len(comp)
    first = {}
    out = np.empty(n, dtype=np.uint64)
    for i in range(n):
        c = comp[i]
        if c not in first:
            first[c] = i
        out[i] = first[c]
    return out


def local_bruteforce(hits, dt: int) -> np.ndarray:
    """Variant (a): components of {(i, j): Chebyshev <= 1 and |dToA| <= dt}."""
    n = len(hits)
    if n == 0:
        return np.empty(0, dtype=np.uint64)
    x = hits["x"].astype(np.int64)
    y = hits["y"].astype(np.int64)
    t = hits["toa"]
    adj_xy = (np.abs(x[:, None] - x[None, :]) <= 1) & (np.abs(y[:, None] - y[None, :]) <= 1)
    # |t_i - t_j| <= dt on uint64 without wrap-around
    big = np.maximum(t[:, None], t[None, :])
    small = np.minimum(t[:, None], t[None, :])
    adj_t = (big - small) <= np.uint64(dt)
    _, comp = connected_components(csr_matrix(adj_xy & adj_t), directed=False)
    return canonical(comp)


def sweep_bruteforce(hits, dt: int, variant: str) -> np.ndarray:
    """Variants (b)/(c) read as Algorithm 1's time sweep: each hit, in
    (toa, index) order, merges every open cluster that has a member on one of
    its 9 pixels.  (b): open iff toa - last <= dt; (c): open iff toa - first <= dt."""
    n = len(hits)
    order = sorted(range(n), key=lambda i: (int(hits["toa"][i]), i))
    clusters = []   # each: dict(members=set, first=int, last=int)
    owner = {}
    for i in order:
        xi, yi, ti = int(hits["x"][i]), int(hits["y"][i]), int(hits["toa"][i])
        hit_clusters = []
        for c in clusters:
            ref = c["last"] if variant == "global" else c["first"]
            if ti - ref > dt:
                continue
            if any(abs(int(hits["x"][m]) - xi) <= 1 and abs(int(hits["y"][m]) - yi) <= 1
                   for m in c["members"]):
                hit_clusters.append(c)
        merged = {"members": {i}, "first": ti, "last": ti}
        for c in hit_clusters:
            merged["members"] |= c["members"]
            merged["first"] = min(merged["first"], c["first"])
            clusters.remove(c)
        clusters.append(merged)
    for ci, c in enumerate(clusters):
        for m in c["members"]:
            owner[m] = ci
    return canonical(np.array([owner[i] for i in range(n)]))


def pixel_ccl(hits, width: int, height: int) -> np.ndarray:
    """Plain 8-connected component labelling of the occupied pixels (the
    textbook frame-based CCL); every hit takes its pixel's component."""
    occ = np.zeros((height, width), dtype=bool)
    occ[hits["y"], hits["x"]] = True
    lab, _ = ndimage.label(occ, structure=np.ones((3, 3), dtype=int))
    return canonical(lab[hits["y"], hits["x"]])


def refines(fine: np.ndarray, coarse: np.ndarray) -> bool:
    """True if every cluster of ``fine`` lies inside one cluster of ``coarse``
    (both canonical label arrays)."""
    fine = np.asarray(fine, dtype=np.int64)
    return bool(np.all(coarse == coarse[fine]))


def random_hits(rng, n, width, height, t_span, tot_max=20):
    from synth import HIT_DTYPE
    h = np.zeros(n, dtype=HIT_DTYPE)
    h["x"] = rng.integers(0, width, n)
    h["y"] = rng.integers(0, height, n)
    h["toa"] = rng.integers(0, t_span + 1, n).astype(np.uint64)
    h["tot"] = rng.integers(1, tot_max + 1, n)
    return h
