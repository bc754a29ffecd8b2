"""Loader for the hand-derived fixtures in ``tests/golden`` (each file cites the
passage of the paper its expected values follow from)."""
import glob
import os

import numpy as np

from oracle import make_hits

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(path):
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.lstrip().startswith("#")]
    w, h, dt = (int(v) for v in rows[0])
    hits, expect, feats = [], {}, []
    for r in rows[1:]:
        if r[0] in ("local", "global", "static"):
            expect[r[0]] = np.array([int(v) for v in r[1:]], dtype=np.uint64)
        elif r[0] == "feature":
            feats.append((int(r[1]), int(r[2]), int(r[3]), int(r[4]), float(r[5]), float(r[6])))
        else:
            hits.append([int(v) for v in r])
    a = np.array(hits, dtype=np.uint64).reshape(-1, 4)
    return {"name": os.path.basename(path), "width": w, "height": h, "dt": dt,
            "hits": make_hits(a[:, 0], a[:, 1], a[:, 2], a[:, 3]),
            "expect": expect, "features": feats}


def all_cases():
    return [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))]
