"""Temporal-split parallel CPU clustering (paper, Sections 3.2-3.3) — a
COMPARISON BASELINE for the benchmark, not the oracle and not the product.

The CUDA library and its binding never import this package.  The method lives in
``tsplit.c`` (C with POSIX threads, compiled with gcc); this module marshals
numpy arrays:

* ``cluster(hits, W, H, dt, window, threads)`` — variant (iii)(a) labels
  (smallest input index per cluster) and per-cluster records ordered by label,
  plus the merge cascade's counters: border cluster pairs examined, cut by
  temporal distance, cut by bounding box, merged after the full check.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HIT_DTYPE = np.dtype([("x", "<u2"), ("y", "<u2"), ("tot", "<u2"),
                      ("reserved", "<u2"), ("toa", "<u8")])
CLUSTER_DTYPE = np.dtype([("label", "<u8"), ("size", "<i8"), ("sum_tot", "<i8"),
                          ("first_toa", "<u8"), ("cx", "<f8"), ("cy", "<f8")])

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsplit.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libtsplit.so")
_lock = threading.Lock()
_lib = None
_ERRORS = {-1: "bad argument", -2: "hit outside the sensor", -3: "out of memory"}
CASCADE_KEYS = ("pairs", "cut_by_time", "cut_by_box", "merged")


def build(force: bool = False) -> str:
    """Compile ``tsplit.c`` into ``_build/libtsplit.so``."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-pthread", "-fPIC", "-shared", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.tsplit_cluster.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p]
        lib.tsplit_cluster.restype = ctypes.c_int
        lib.tsplit_hit_size.restype = ctypes.c_uint32
        lib.tsplit_cluster_size.restype = ctypes.c_uint32
        assert lib.tsplit_hit_size() == HIT_DTYPE.itemsize
        assert lib.tsplit_cluster_size() == CLUSTER_DTYPE.itemsize
        _lib = lib
    return _lib


def cluster(hits, width: int, height: int, dt: int, window: int = 6400, threads: int | None = None):
    """Labels, records ordered by label, and the cascade counters (a dict).

    ``window`` is the split window in ToA ticks (6400 ticks = 10 us at
    1.5625 ns, the paper's example); it must exceed ``dt``.  ``threads``
    defaults to the host's cores."""
    h = np.ascontiguousarray(hits)
    if h.dtype != HIT_DTYPE:
        raise TypeError(f"hits must have dtype {HIT_DTYPE}")
    n = len(h)
    if threads is None:
        threads = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    lab = np.empty(n, dtype=np.uint64)
    rec = np.empty(max(n, 1), dtype=CLUSTER_DTYPE)
    m = ctypes.c_uint64(0)
    cascade = np.zeros(4, dtype=np.uint64)
    rc = _load().tsplit_cluster(h.ctypes.data if n else None, n, width, height, dt, window,
                                int(threads), lab.ctypes.data if n else None, rec.ctypes.data,
                                ctypes.byref(m), cascade.ctypes.data)
    if rc != 0:
        raise ValueError(f"tsplit: {_ERRORS.get(rc, rc)}")
    return lab, rec[: m.value].copy(), dict(zip(CASCADE_KEYS, (int(v) for v in cascade)))
