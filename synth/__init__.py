"""Seeded synthetic Timepix hit streams (inputs only, no clustering arithmetic).

The paper benchmarks on beam-test datasets (Am-241 photons, 40 GeV/c pions,
385 GeV/c lead ions; Section 4, table of cluster sizes) that are not
available here.  These generators stand in for them with the workload shapes
of the five benchmark configurations:

* ``cfg0``: 256x256 sensor, 1M hits, blobs only, events at 1 Mevent/s.
* ``cfg1``: 256x256 sensor, 64M hits at 40 Mhits/s, 80 % blobs / 20 % tracks,
  dead-time refires.
* ``cfg2``: 16 detectors (ten 256x256, six 448x512), chunks log-uniform in
  [1e4, 8e6] hits, about 40M hits in total, rates log-uniform in [5, 80] Mhits/s.
* ``cfg3``: 8 streams at 50 Mhits/s each, cut into chunks log-uniform in
  [64k, 2M] hits.
* ``cfg4``: 448x512 sensor, 512M hits at 2.5 Ghits/s, config-1 mix.

The hit record is 16 bytes: ``x, y, tot, reserved`` as uint16 and ``toa`` as
uint64 in 1.5625 ns ticks.  Both the CPU oracle and the CUDA path read these
arrays; nothing here depends on either of them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HIT_DTYPE = np.dtype([("x", "<u2"), ("y", "<u2"), ("tot", "<u2"),
                      ("reserved", "<u2"), ("toa", "<u8")])
assert HIT_DTYPE.itemsize == 16

TICKS_PER_SECOND = 6.4e8          # 1 tick = 1.5625 ns
DT_200NS = 128                    # 200 ns, the default time window
DT_600NS = 384                    # 600 ns

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hitgen.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libhitgen.so")
_lock = threading.Lock()
_lib = None


class _Params(ctypes.Structure):
    _fields_ = [("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("n", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("event_rate", ctypes.c_double), ("hit_rate", ctypes.c_double),
                ("track_frac", ctypes.c_double),
                ("track_min", ctypes.c_uint32), ("track_max", ctypes.c_uint32),
                ("max_gradient", ctypes.c_double),
                ("toa_jitter", ctypes.c_uint32), ("blob_p", ctypes.c_double),
                ("tot_mean", ctypes.c_double), ("tot_max", ctypes.c_uint32),
                ("dead_time", ctypes.c_uint32), ("shuffle_window", ctypes.c_uint32),
                ("t0", ctypes.c_uint64)]


def build(force: bool = False) -> str:
    """Compile ``hitgen.c`` into ``_build/libhitgen.so`` (gcc, portable flags)."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                        "-ffp-contract=off", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.hitgen_generate.argtypes = [ctypes.POINTER(_Params), ctypes.c_void_p,
                                        ctypes.POINTER(ctypes.c_uint64)]
        lib.hitgen_generate.restype = ctypes.c_int
        lib.hitgen_params_size.restype = ctypes.c_uint32
        assert lib.hitgen_params_size() == ctypes.sizeof(_Params)
        _lib = lib
    return _lib


def generate(width: int, height: int, n: int, seed: int, *, event_rate_hz: float = 0.0,
             hit_rate_hz: float = 0.0, track_frac: float = 0.0, track_min: int = 10,
             track_max: int = 300, max_gradient: float = 20.0, toa_jitter: int = 64,
             blob_p: float = 0.3, tot_mean: float = 40.0, tot_max: int = 1023,
             dead_time: bool = False, shuffle_window: int = 1000,
             t0: int = 1_000_000) -> tuple[np.ndarray, int]:
    """Draw ``n`` hits.  Returns ``(hits, t)`` where ``t`` is the smallest
    constant for which the stream is t-ordered (toa[i] < toa[j] + t, i < j)."""
    if event_rate_hz <= 0 and hit_rate_hz <= 0:
        raise ValueError("need event_rate_hz or hit_rate_hz")
    p = _Params(width, height, n, seed, event_rate_hz / TICKS_PER_SECOND,
                hit_rate_hz / TICKS_PER_SECOND, track_frac, track_min, track_max,
                max_gradient, toa_jitter, blob_p, tot_mean, tot_max, int(dead_time),
                shuffle_window, t0)
    out = np.empty(n, dtype=HIT_DTYPE)
    t = ctypes.c_uint64(0)
    rc = _load().hitgen_generate(ctypes.byref(p), out.ctypes.data if n else None,
                                 ctypes.byref(t))
    if rc != 0:
        raise RuntimeError(f"hitgen_generate failed ({rc})")
    return out, int(t.value)


# ---------------------------------------------------------------------------
# the benchmark configurations

def cfg0(scale: float = 1.0, seed: int = 0):
    """256x256, 1M hits, random-walk blobs, 1 Mevent/s, window-shuffled."""
    n = max(1, int(1_000_000 * scale))
    return generate(256, 256, n, seed, event_rate_hz=1e6)


def cfg1(scale: float = 1.0, seed: int = 1000, width: int = 256, height: int = 256,
         hit_rate_hz: float = 40e6, tot_max: int = 1023):
    """256x256, 64M hits at 40 Mhits/s, 20 % tracks, dead-time refires."""
    n = max(1, int(64 * 2**20 * scale))
    return generate(width, height, n, seed, hit_rate_hz=hit_rate_hz, track_frac=0.2,
                    dead_time=True, tot_max=tot_max)


def generate_blocked(width: int, height: int, n: int, seed: int, blocks: int,
                     **kw) -> tuple[np.ndarray, int]:
    """``n`` hits drawn as ``blocks`` consecutive, independently seeded
    sub-streams, generated in parallel host threads (the C generator is
    sequential, about 0.4 us per hit; half a billion hits would take minutes
    on one core).  Block k uses seed ``seed * 1000003 + k + 1`` and follows
    block k - 1 in time after a quiet gap of 2048 ticks, longer than any
    ToT (<= 1023, so no pixel is still busy across a block border) and than
    the window shuffle's reach, so the concatenation is t-ordered with the
    largest t of its blocks.  Statistically it is the same workload; it is
    not the same stream as ``generate`` with one seed."""
    if blocks <= 1:
        return generate(width, height, n, seed, **kw)
    sizes = [n // blocks + (1 if k < n % blocks else 0) for k in range(blocks)]
    parts: list = [None] * blocks
    errors: list = []

    def work(k):
        try:
            parts[k] = generate(width, height, sizes[k], seed * 1000003 + k + 1, **kw)
        except Exception as e:   # re-raised below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(k,)) for k in range(blocks)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    if errors:
        raise errors[0]
    out = np.empty(n, dtype=HIT_DTYPE)
    t_max, pos, shift = 1, 0, 0
    t0 = kw.get("t0", 1_000_000)
    for hits, t in parts:
        m = len(hits)
        out[pos:pos + m] = hits
        if m:
            out["toa"][pos:pos + m] += np.uint64(shift)
            shift += int(hits["toa"].max()) - t0 + 2048
        pos += m
        t_max = max(t_max, t)
    return out, t_max


def cfg4(scale: float = 1.0, seed: int = 4000, blocks: int = 1):
    """448x512 (Timepix4), 512M hits at 2.5 Ghits/s, config-1 mix, ToT <= 1023.
    ``blocks > 1`` draws it as that many consecutive independently seeded
    sub-streams in parallel (``generate_blocked``), for the full size."""
    n = max(1, int(512 * 2**20 * scale))
    return generate_blocked(448, 512, n, seed, blocks, hit_rate_hz=2.5e9, track_frac=0.2,
                            dead_time=True, tot_max=1023)


def log_uniform_sizes(rng: np.random.Generator, lo: float, hi: float, total: int) -> list[int]:
    """Chunk sizes drawn log-uniformly in [lo, hi] until their sum reaches ``total``."""
    sizes, s = [], 0
    while s < total:
        c = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        c = min(c, total - s) if s + c > total else c
        sizes.append(max(1, c))
        s += sizes[-1]
    return sizes


def cfg2(scale: float = 1.0, seed: int = 2000):
    """16 detectors (10 x 256x256, 6 x 448x512).  Returns a list of
    ``(width, height, hits, chunk_sizes, t)`` per detector."""
    rng = np.random.default_rng(seed)
    geoms = [(256, 256)] * 10 + [(448, 512)] * 6
    total = max(16, int(40_000_000 * scale))
    lo, hi = max(1.0, 1e4 * scale), max(2.0, 8e6 * scale)
    chunks = log_uniform_sizes(rng, lo, hi, total)
    per_det: list[list[int]] = [[] for _ in geoms]
    for i, c in enumerate(chunks):
        per_det[i % len(geoms)].append(c)
    rates = np.exp(rng.uniform(np.log(5e6), np.log(80e6), size=len(geoms)))
    out = []
    for d, ((w, h), sizes) in enumerate(zip(geoms, per_det)):
        n = int(sum(sizes))
        hits, t = generate(w, h, n, seed * 100 + d, hit_rate_hz=float(rates[d]),
                           track_frac=0.2, dead_time=True) if n else (np.empty(0, HIT_DTYPE), 1)
        out.append((w, h, hits, sizes, t))
    return out


def cfg3(hits_per_stream: int, n_streams: int = 8, seed: int = 3000,
         chunk_lo: int = 65536, chunk_hi: int = 2 * 2**20, rate_hz: float = 50e6):
    """Serving: ``n_streams`` 256x256 streams at ``rate_hz`` each, each cut into
    chunks log-uniform in [chunk_lo, chunk_hi] hits.  Returns a list of
    ``(hits, chunk_sizes, t)`` per stream."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_streams):
        hits, t = generate(256, 256, hits_per_stream, seed * 100 + s, hit_rate_hz=rate_hz,
                           track_frac=0.2, dead_time=True)
        sizes = log_uniform_sizes(rng, chunk_lo, chunk_hi, hits_per_stream)
        out.append((hits, sizes, t))
    return out
