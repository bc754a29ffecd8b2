"""The oracle's pins catch plausible mistakes: each mistake below is planted
in a copy of the oracle's C source (never the committed file), the copy is
compiled, and the oracle pin suites (tests/test_oracle.py and
tests/test_oracle_filling.py) must fail on it."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "tpc_oracle.c")

MISTAKES = {
    "strict time window": ("return (a >= b ? a - b : b - a) <= dt;",
                           "return (a >= b ? a - b : b - a) < dt;"),
    "4-connectivity": ("for (int dx = -1; dx <= 1; ++dx) {\n                    int64_t px",
                       "for (int dx = -1; dx <= 1; ++dx) { if (dx && dy) continue;\n                    int64_t px"),
    "(b) open test on the first ToA": ("uint64_t ref = mode == 1 ? u.last[r] : u.first[r];",
                                       "uint64_t ref = mode == 1 ? u.first[r] : u.first[r];"),
    "open test off by one": ("if (t - ref > dt) continue;", "if (t - ref >= dt) continue;"),
    "centroid x from y sums": ("out[c].cx = (double)swx[c] / w;", "out[c].cx = (double)swy[c] / w;"),
    "label not the smallest index": ("if (label[v] == NONE) { label[v] = s;",
                                     "if (label[v] == NONE) { label[v] = u;"),
    "own pixel not a neighbour": (
        "                pix_vec *pv = &pix[(uint64_t)py * W + (uint64_t)px];",
        "                if (!dx && !dy) continue; pix_vec *pv = &pix[(uint64_t)py * W + (uint64_t)px];"),
    "merged cluster keeps one first ToA": (
        "uint64_t f = u.first[r] < u.first[root] ? u.first[r] : u.first[root];",
        "uint64_t f = u.first[r];"),
    "centroid weights missing": ("swx[c] += (uint64_t)h[i].tot * h[i].x;", "swx[c] += (uint64_t)h[i].x;"),
    "ToA search window one tick short": ("uint64_t t_lo = t >= dt ? t - dt : 0;",
                                         "uint64_t t_lo = t >= dt ? t - dt + 1 : 0;"),
    "pixel lists not in ToA order": ("if (ti != tj) return ti < tj ? -1 : 1;", "if (0) return 0;"),
    "first ToA taken as the largest": ("if (h[i].toa < out[c].first_toa) out[c].first_toa = h[i].toa;",
                                       "if (h[i].toa > out[c].first_toa || out[c].first_toa == UINT64_MAX) "
                                       "out[c].first_toa = h[i].toa;"),
    "centroid y weighted by x": ("swy[c] += (uint64_t)h[i].tot * h[i].y;", "swy[c] += (uint64_t)h[i].tot * h[i].x;"),
    "cut without the closing slack": ("cut[cur] = sat_add(toa_max, t_closing);   /* sendToDevice(buffer) */",
                                      "cut[cur] = toa_max;   /* sendToDevice(buffer) */"),
    "late hits kept in a full buffer": ("            buffer_of[i] = cur + 1;\n            size_next++;",
                                        "            buffer_of[i] = cur;\n            size_cur++;"),
    "closing time inclusive": ("} else if (toa < sat_add(toa_max, t_closing) && size_cur < b) {",
                               "} else if (toa <= sat_add(toa_max, t_closing) && size_cur < b) {"),
    "toa_max not kept while filling": ("if (toa > toa_max) toa_max = toa;", ";"),
    "send trigger without the disorder bound": ("toa - toa_max > sat_add(t, t_closing)",
                                                "toa - toa_max > t_closing"),
    "closing phase without room check": ("if (size_cur < b - b_t) {", "if (size_cur < b) {"),
}
PIN_FILES = ["test_oracle.py", "test_oracle_filling.py"]


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_pins_catch_planted_mistake(name, tmp_path):
    good, bad = MISTAKES[name]
    src = open(SRC).read()
    assert src.count(good) == 1, "the mistake's site moved: update this test"
    mutant = tmp_path / "tpc_oracle.c"
    mutant.write_text(src.replace(good, bad))
    env = dict(os.environ, TPC_ORACLE_SRC=str(mutant), TPC_ORACLE_BUILD=str(tmp_path / "build"))
    out = subprocess.run([sys.executable, "-m", "pytest",
                          *[os.path.join(ROOT, "tests", f) for f in PIN_FILES],
                          "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode != 0, f"planted mistake '{name}' passed every pin:\n{out.stdout[-2000:]}"
