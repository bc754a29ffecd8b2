"""CPU oracle for Timepix hit clustering — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (the CUDA library and its
binding) never calls it and shares no code with it.

The arithmetic lives in ``tpc_oracle.c`` (plain sequential C, compiled with
gcc); this module only marshals numpy arrays:

* ``labels(hits, W, H, dt, variant)`` — canonical labels (smallest input index
  per cluster) for variant ``"local"`` (a), ``"global"`` (b) or ``"static"`` (c)
  of the paper's cluster definition (Section 2, conditions (i)-(iii)).
* ``features(hits, labels)`` — per-cluster size, sum ToT, first ToA and the
  ToT-weighted centroid (fp64), ordered by label.
* ``fill_buffers(hits, b, b_t, t, t_closing)`` — the host-side hit buffer
  filling of Algorithm 2: which buffer each hit is sent in.
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
# TPC_ORACLE_SRC / TPC_ORACLE_BUILD point the oracle at another copy of its
# source (tests/test_oracle_mutations.py plants mistakes in such copies to show
# that the pins catch them); unset, the committed source is used.
_SRC = os.environ.get("TPC_ORACLE_SRC") or os.path.join(_HERE, "tpc_oracle.c")
_BUILD = os.environ.get("TPC_ORACLE_BUILD") or os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libtpc_oracle.so")
_lock = threading.Lock()
_lib = None

_ERRORS = {-1: "bad argument", -2: "hit outside the sensor", -3: "out of memory"}


def build(force: bool = False) -> str:
    """Compile ``tpc_oracle.c`` into ``_build/libtpc_oracle.so``."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC],
                       check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        for name in ("oracle_labels_local", "oracle_labels_global", "oracle_labels_static"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                          ctypes.c_uint64, ctypes.c_void_p]
            f.restype = ctypes.c_int
        lib.oracle_features.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)]
        lib.oracle_features.restype = ctypes.c_int
        lib.oracle_fill_buffers.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_uint64)]
        lib.oracle_fill_buffers.restype = ctypes.c_int
        lib.oracle_hit_size.restype = ctypes.c_uint32
        lib.oracle_cluster_size.restype = ctypes.c_uint32
        assert lib.oracle_hit_size() == HIT_DTYPE.itemsize
        assert lib.oracle_cluster_size() == CLUSTER_DTYPE.itemsize
        _lib = lib
    return _lib


def _as_hits(hits) -> np.ndarray:
    h = np.ascontiguousarray(hits)
    if h.dtype != HIT_DTYPE:
        raise TypeError(f"hits must have dtype {HIT_DTYPE}")
    return h


VARIANTS = {"local": "oracle_labels_local", "global": "oracle_labels_global",
            "static": "oracle_labels_static", 0: "oracle_labels_local",
            1: "oracle_labels_global", 2: "oracle_labels_static"}


def labels(hits, width: int, height: int, dt: int, variant="local") -> np.ndarray:
    """Canonical cluster labels (uint64, smallest input index per cluster)."""
    h = _as_hits(hits)
    n = len(h)
    out = np.empty(n, dtype=np.uint64)
    fn = getattr(_load(), VARIANTS[variant])
    rc = fn(h.ctypes.data if n else None, n, width, height, dt,
            out.ctypes.data if n else None)
    if rc != 0:
        raise ValueError(f"oracle: {_ERRORS.get(rc, rc)}")
    return out


def features(hits, lab) -> np.ndarray:
    """Per-cluster records ordered by label (see ``CLUSTER_DTYPE``)."""
    h = _as_hits(hits)
    lab = np.ascontiguousarray(lab, dtype=np.uint64)
    n = len(h)
    out = np.empty(max(n, 1), dtype=CLUSTER_DTYPE)
    m = ctypes.c_uint64(0)
    rc = _load().oracle_features(h.ctypes.data if n else None, n,
                                 lab.ctypes.data if n else None, out.ctypes.data,
                                 ctypes.byref(m))
    if rc != 0:
        raise ValueError(f"oracle: {_ERRORS.get(rc, rc)}")
    return out[: m.value].copy()


def fill_buffers(hits, b: int, b_t: int, t: int, t_closing: int):
    """Algorithm 2 (hit buffer filling) over the hits in arrival order.

    Returns ``(buffer_of, cut)``: the number of the buffer each hit lands in
    (buffers numbered in the order they are sent) and, per buffer, the closing
    time ``toa_max + t_closing`` at which it was sent (``2**64 - 1`` for the
    buffers sent at the end of the stream)."""
    h = _as_hits(hits)
    n = len(h)
    buffer_of = np.empty(n, dtype=np.uint64)
    cut = np.empty(n + 1, dtype=np.uint64)
    m = ctypes.c_uint64(0)
    rc = _load().oracle_fill_buffers(h.ctypes.data if n else None, n, b, b_t, t, t_closing,
                                     buffer_of.ctypes.data if n else None, cut.ctypes.data,
                                     ctypes.byref(m))
    if rc != 0:
        raise ValueError(f"oracle: {_ERRORS.get(rc, rc)}")
    return buffer_of, cut[: m.value].copy()


def make_hits(x, y, toa, tot=None) -> np.ndarray:
    """Pack coordinate/time arrays into the 16-byte hit record."""
    x = np.asarray(x)
    h = np.zeros(len(x), dtype=HIT_DTYPE)
    h["x"] = x
    h["y"] = np.asarray(y)
    h["toa"] = np.asarray(toa)
    h["tot"] = 1 if tot is None else np.asarray(tot)
    return h
