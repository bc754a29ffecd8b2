"""Thin ctypes binding of libtpc (the C ABI declared in include/tpc.h).

Argument marshalling only: every step of the clustering runs in the CUDA
library.  There is no CPU fallback — if libtpc.so is missing the import of a
Clusterer fails loudly.  Device memory and streams come from PyTorch when
device tensors are passed; host data are numpy arrays.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HIT_DTYPE = np.dtype([("x", "<u2"), ("y", "<u2"), ("tot", "<u2"),
                      ("reserved", "<u2"), ("toa", "<u8")])
CLUSTER_DTYPE = np.dtype([("label", "<u8"), ("size", "<i8"), ("sum_tot", "<i8"),
                          ("first_toa", "<u8"), ("cx", "<f4"), ("cy", "<f4")])
SNAPSHOT_HEADER_DTYPE = np.dtype([("magic", "<u4"), ("version", "<u4"), ("width", "<u4"),
                                  ("height", "<u4"), ("dt", "<u8"), ("max_disorder", "<u8"),
                                  ("pushed", "<u8"), ("seen_max", "<u8"), ("watermark", "<u8"),
                                  ("has_seen", "<u4"), ("n_carry", "<u4")])
assert HIT_DTYPE.itemsize == 16 and CLUSTER_DTYPE.itemsize == 40
assert SNAPSHOT_HEADER_DTYPE.itemsize == 64

TPC_HOST, TPC_DEVICE = 0, 1
VARIANTS = {"local": 0, "global": 1, "static": 2, 0: 0, 1: 1, 2: 2}
OPT_MAX_DISORDER, OPT_MEM_BUDGET, OPT_STREAM, OPT_CTAS_PER_SM, OPT_FAIL_ALLOC = 1, 2, 3, 4, 5

STATUS = {0: "TPC_OK", -1: "TPC_ERR_ARG", -2: "TPC_ERR_RANGE", -3: "TPC_ERR_NOMEM",
          -4: "TPC_ERR_BUSY", -5: "TPC_ERR_TIMEOUT", -6: "TPC_ERR_CUDA", -7: "TPC_ERR_CAP",
          -8: "TPC_ERR_SPAN", -9: "TPC_ERR_LATE", -10: "TPC_ERR_STATE"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libtpc.so")

# every entry point of include/tpc.h with its ctypes signature
_VP, _SZ, _U64, _U32, _INT = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
SIGNATURES = {
    "tpc_create": ([_U32, _U32, _U64, _INT, ctypes.POINTER(_VP)], _INT),
    "tpc_set_option": ([_VP, _INT, _U64], _INT),
    "tpc_push": ([_VP, _VP, _SZ, _INT], _INT),
    "tpc_flush": ([_VP], _INT),
    "tpc_sync": ([_VP], _INT),
    "tpc_labels": ([_VP, _VP, _VP, _SZ, ctypes.POINTER(_SZ), _INT], _INT),
    "tpc_labels_async": ([_VP, _VP, _SZ, ctypes.POINTER(_SZ), _INT], _INT),
    "tpc_cluster_features": ([_VP, _VP, _SZ, ctypes.POINTER(_SZ), _INT], _INT),
    "tpc_batch_flush": ([ctypes.POINTER(_VP), _INT], _INT),
    "tpc_counts": ([_VP, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)], _INT),
    "tpc_device_bytes": ([_VP, ctypes.POINTER(_SZ)], _INT),
    "tpc_forest": ([_VP, _VP, _VP, _SZ, ctypes.POINTER(_SZ)], _INT),
    "tpc_profile_flush": ([_VP, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_float),
                           _INT, ctypes.POINTER(_INT)], _INT),
    "tpc_snapshot": ([_VP, _VP, _SZ, ctypes.POINTER(_SZ)], _INT),
    "tpc_restore": ([_VP, _VP, _SZ], _INT),
    "tpc_cluster_static": ([_VP, _SZ, _U32, _U32, _U64, _VP, _VP, _SZ, _VP, _VP], _INT),
    "tpc_filler_create": ([_U64, _U64, _U64, _U64, ctypes.POINTER(_VP)], _INT),
    "tpc_filler_store": ([_VP, _VP, _SZ], _INT),
    "tpc_filler_finish": ([_VP], _INT),
    "tpc_filler_ready": ([_VP, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)], _INT),
    "tpc_filler_take": ([_VP, _VP, _VP, _SZ, ctypes.POINTER(_SZ), ctypes.POINTER(_U64)], _INT),
    "tpc_filler_send": ([_VP, _VP, _VP, _SZ, ctypes.POINTER(_SZ), ctypes.POINTER(_U64)], _INT),
    "tpc_filler_destroy": ([_VP], None),
    "tpc_server_create": ([_U64, ctypes.POINTER(_VP)], _INT),
    "tpc_server_add_stream": ([_VP, _U32, _U32, _U64, _U64, ctypes.POINTER(_INT)], _INT),
    "tpc_server_submit": ([_VP, _INT, _VP, _SZ, _VP, _VP, _VP, _SZ, _U64, _INT], _INT),
    "tpc_server_wait": ([_VP, _VP, ctypes.c_int64], _INT),
    "tpc_server_stats_get": ([_VP, _VP], _INT),
    "tpc_server_destroy": ([_VP], None),
    "tpc_set_tuning": ([_VP, _VP], _INT),
    "tpc_get_tuning": ([_VP, _VP], _INT),
    "tpc_tune_batch": ([ctypes.POINTER(_VP), _INT, ctypes.c_char_p, _INT, _VP], _INT),
    "tpc_tune_cache_lookup": ([ctypes.c_char_p, ctypes.c_char_p, _VP, ctypes.POINTER(ctypes.c_double)], _INT),
    "tpc_tune_cache_store": ([ctypes.c_char_p, ctypes.c_char_p, _VP, ctypes.c_double], _INT),
    "tpc_variant_stats_get": ([_VP, _VP], _INT),
    "tpc_bind_outputs": ([_VP, _VP, _VP, _SZ], _INT),
    "tpc_strerror": ([_INT], ctypes.c_char_p),
    "tpc_destroy": ([_VP], None),
}

_lib = None


class Tuning(ctypes.Structure):
    """``tpc_tuning``: launch choices (results never depend on them)."""
    _fields_ = [("ctas_sort", ctypes.c_uint8), ("ctas_link", ctypes.c_uint8),
                ("ctas_acc", ctypes.c_uint8), ("ctas_out", ctypes.c_uint8),
                ("acc_span", ctypes.c_uint16), ("general_link", ctypes.c_uint8),
                ("order", ctypes.c_uint8)]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


class TuneReport(ctypes.Structure):
    """``tpc_tune_report``."""
    _fields_ = [("chosen", Tuning), ("from_cache", ctypes.c_uint32), ("trials", ctypes.c_uint32),
                ("untuned_ms", ctypes.c_double), ("tuned_ms", ctypes.c_double),
                ("key", ctypes.c_char * 192)]


assert ctypes.sizeof(Tuning) == 8 and ctypes.sizeof(TuneReport) == 224


class TpcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        msg = _lib.tpc_strerror(status).decode() if _lib is not None else self.name
        super().__init__(f"{what}: {self.name} ({msg})" if what else f"{self.name} ({msg})")


def load_library(path: str = LIB_PATH):
    """Load libtpc.so and declare its signatures.  Raises if it is not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libtpc.so not found at {path}: build it with "
                               "paper_2412_11809_gb300.build.build() (needs nvcc)")
        lib = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        raise TpcError(rc, what)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _device_hits(t):
    """(pointer, n) of a contiguous CUDA tensor holding 16-byte hit records."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device hits must be a contiguous CUDA tensor")
    nbytes = t.numel() * t.element_size()
    if nbytes % 16:
        raise ValueError("device hits must hold whole 16-byte records")
    return t.data_ptr(), nbytes // 16


class Clusterer:
    """One clustering context (one sensor / stream), see ``tpc_create``."""

    def __init__(self, width: int, height: int, dt: int, variant="local", *,
                 max_disorder: int | None = None, mem_budget: int | None = None,
                 stream=None, ctas_per_sm: int | None = None):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.tpc_create(width, height, dt, VARIANTS[variant], ctypes.byref(h)), "tpc_create")
        self._h = h
        self._lib = lib
        self._keep = []          # device inputs that must outlive the queued work
        self._own_stream = stream is None
        self.width, self.height, self.dt = width, height, dt
        if stream is not None:
            raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
            _check(lib.tpc_set_option(h, OPT_STREAM, raw), "stream")
        if mem_budget is not None:
            _check(lib.tpc_set_option(h, OPT_MEM_BUDGET, mem_budget), "mem_budget")
        if ctas_per_sm is not None:
            _check(lib.tpc_set_option(h, OPT_CTAS_PER_SM, ctas_per_sm), "ctas_per_sm")
        if max_disorder is not None:
            _check(lib.tpc_set_option(h, OPT_MAX_DISORDER, max_disorder), "max_disorder")

    @property
    def handle(self):
        return self._h

    def set_option(self, key: int, value: int):
        """``tpc_set_option`` (see ``tpc_option``; e.g. ``OPT_MAX_DISORDER``)."""
        _check(self._lib.tpc_set_option(self._h, key, value), "tpc_set_option")

    def inject_alloc_failure(self, nth: int):
        """Test hook: the nth allocation from now fails as an out-of-memory
        would (``TPC_OPT_FAIL_ALLOC``); 0 turns it off."""
        self.set_option(OPT_FAIL_ALLOC, nth)

    def push(self, hits):
        """Append a chunk: a numpy array of HIT_DTYPE (host) or a CUDA tensor."""
        if _is_torch(hits):
            ptr, n = _device_hits(hits)
            self._keep.append(hits)
            if self._own_stream:
                # the context's stream does not order after torch's: let the
                # producer of `hits` finish first
                import torch
                torch.cuda.current_stream(hits.device).synchronize()
            _check(self._lib.tpc_push(self._h, ptr, n, TPC_DEVICE), "tpc_push")
        else:
            a = np.ascontiguousarray(hits)
            if a.dtype != HIT_DTYPE:
                raise TypeError(f"host hits must have dtype {HIT_DTYPE}")
            _check(self._lib.tpc_push(self._h, a.ctypes.data if len(a) else None, len(a), TPC_HOST),
                   "tpc_push")

    def push_ptr(self, ptr: int, n: int, device: bool):
        """Append n hits from a raw pointer (host or device memory)."""
        _check(self._lib.tpc_push(self._h, ptr, n, TPC_DEVICE if device else TPC_HOST), "tpc_push")

    def flush(self):
        _check(self._lib.tpc_flush(self._h), "tpc_flush")

    def labels_into(self, labels_ptr: int, cap: int, device: bool, indices_ptr: int | None = None) -> int:
        """Write the last step's labels into caller memory; returns the count."""
        n_out = ctypes.c_size_t()
        rc = self._lib.tpc_labels(self._h, labels_ptr, indices_ptr, cap, ctypes.byref(n_out),
                                  TPC_DEVICE if device else TPC_HOST)
        self._keep.clear()
        _check(rc, "tpc_labels")
        return n_out.value

    def labels_async(self, labels_ptr: int, cap: int, device: bool) -> int:
        """Queue the copy of the last one-shot step's labels (valid after sync()
        or the next retrieval); returns their count."""
        n_out = ctypes.c_size_t()
        _check(self._lib.tpc_labels_async(self._h, labels_ptr, cap, ctypes.byref(n_out),
                                          TPC_DEVICE if device else TPC_HOST), "tpc_labels_async")
        return n_out.value

    def features_into(self, rec_ptr: int, cap: int, device: bool) -> int:
        """Write the last step's cluster records into caller memory; returns the count."""
        n_out = ctypes.c_size_t()
        _check(self._lib.tpc_cluster_features(self._h, rec_ptr, cap, ctypes.byref(n_out),
                                              TPC_DEVICE if device else TPC_HOST), "features")
        return n_out.value

    def sync(self):
        rc = self._lib.tpc_sync(self._h)
        self._keep.clear()
        _check(rc, "tpc_sync")

    def counts(self) -> tuple[int, int, int]:
        a, b, c = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
        _check(self._lib.tpc_counts(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "tpc_counts")
        return a.value, b.value, c.value

    def labels(self, device: bool = False, with_indices: bool = False):
        """Labels finalised by the last step (uint64 numpy, or int64 CUDA tensor)."""
        n, _, _ = self.counts()
        n_out = ctypes.c_size_t()
        if device:
            import torch
            lab = torch.empty(n, dtype=torch.int64, device="cuda")
            idx = torch.empty(n, dtype=torch.int64, device="cuda") if with_indices else None
            _check(self._lib.tpc_labels(self._h, lab.data_ptr() if n else None,
                                        idx.data_ptr() if (idx is not None and n) else None,
                                        n, ctypes.byref(n_out), TPC_DEVICE), "tpc_labels")
        else:
            lab = np.empty(n, dtype=np.uint64)
            idx = np.empty(n, dtype=np.uint64) if with_indices else None
            _check(self._lib.tpc_labels(self._h, lab.ctypes.data if n else None,
                                        idx.ctypes.data if (idx is not None and n) else None,
                                        n, ctypes.byref(n_out), TPC_HOST), "tpc_labels")
        self._keep.clear()
        return (lab, idx) if with_indices else lab

    def features(self, device: bool = False):
        """Cluster records finalised by the last step, ordered by label."""
        _, m, _ = self.counts()
        n_out = ctypes.c_size_t()
        if device:
            import torch
            rec = torch.empty((m, CLUSTER_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
            _check(self._lib.tpc_cluster_features(self._h, rec.data_ptr() if m else None, m,
                                                  ctypes.byref(n_out), TPC_DEVICE), "features")
        else:
            rec = np.empty(m, dtype=CLUSTER_DTYPE)
            _check(self._lib.tpc_cluster_features(self._h, rec.ctypes.data if m else None, m,
                                                  ctypes.byref(n_out), TPC_HOST), "features")
        return rec

    def profile_flush(self) -> list[tuple[str, float]]:
        """Like flush(), kernels launched one by one; returns (kernel, ms) in order."""
        cap = 64
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_float * cap)()
        n = ctypes.c_int()
        _check(self._lib.tpc_profile_flush(self._h, names, ms, cap, ctypes.byref(n)),
               "tpc_profile_flush")
        return [(names[i].decode(), float(ms[i])) for i in range(n.value)]

    def snapshot(self) -> bytes:
        """Checkpoint of a streaming context's open state (``tpc_snapshot``)."""
        n = ctypes.c_size_t()
        rc = self._lib.tpc_snapshot(self._h, None, 0, ctypes.byref(n))
        if rc != -7:   # TPC_ERR_CAP: the size query
            _check(rc, "tpc_snapshot")
        buf = ctypes.create_string_buffer(n.value)
        _check(self._lib.tpc_snapshot(self._h, buf, n.value, ctypes.byref(n)), "tpc_snapshot")
        return buf.raw[:n.value]

    def restore(self, snap: bytes):
        """Continue the stream a snapshot was taken of (``tpc_restore``)."""
        buf = ctypes.create_string_buffer(bytes(snap), len(snap))
        _check(self._lib.tpc_restore(self._h, buf, len(snap)), "tpc_restore")
        self._keep.clear()

    def forest(self):
        """Diagnostics (``tpc_forest``): the last step's union-find forest as
        (parent, input_pos) uint32 arrays indexed by (ToA, input) position."""
        n = ctypes.c_size_t()
        rc = self._lib.tpc_forest(self._h, None, None, 0, ctypes.byref(n))
        if rc not in (0, -7):   # TPC_ERR_CAP: the size query
            _check(rc, "tpc_forest")
        parent = np.empty(n.value, dtype=np.uint32)
        pos = np.empty(n.value, dtype=np.uint32)
        _check(self._lib.tpc_forest(self._h, parent.ctypes.data if n.value else None,
                                    pos.ctypes.data if n.value else None, n.value,
                                    ctypes.byref(n)), "tpc_forest")
        return parent, pos

    def set_tuning(self, tuning: "Tuning | dict | None"):
        """``tpc_set_tuning``: a Tuning, a dict of its fields, or None (defaults)."""
        if isinstance(tuning, dict):
            tuning = Tuning(**tuning)
        _check(self._lib.tpc_set_tuning(self._h, None if tuning is None else ctypes.byref(tuning)),
               "tpc_set_tuning")

    def tuning(self) -> Tuning:
        t = Tuning()
        _check(self._lib.tpc_get_tuning(self._h, ctypes.byref(t)), "tpc_get_tuning")
        return t

    def bind_outputs(self, labels_ptr: int | None, records_ptr: int | None, cap: int = 0):
        """``tpc_bind_outputs``: device buffers every following one-shot step
        writes its labels and records into (None, None unbinds)."""
        _check(self._lib.tpc_bind_outputs(self._h, labels_ptr, records_ptr, cap), "tpc_bind_outputs")

    def variant_stats(self) -> dict:
        """``tpc_variant_stats_get``: diagnostics of the last (b)/(c) flush."""
        st = (ctypes.c_uint32 * 7)()
        _check(self._lib.tpc_variant_stats_get(self._h, st), "tpc_variant_stats_get")
        return dict(zip(("rounds", "full_rounds", "exact_checks", "windowed", "window_fallbacks",
                         "global_sweeps", "first_open_edges"), st))

    def device_bytes(self) -> int:
        b = ctypes.c_size_t()
        _check(self._lib.tpc_device_bytes(self._h, ctypes.byref(b)), "tpc_device_bytes")
        return b.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tpc_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def batch_flush(clusterers) -> None:
    """Cluster the pending hits of several contexts in one batched step."""
    lib = load_library()
    arr = (ctypes.c_void_p * len(clusterers))(*[c.handle.value for c in clusterers])
    _check(lib.tpc_batch_flush(arr, len(clusterers)), "tpc_batch_flush")


def tune_batch(clusterers, cache_path: str | None = None, force: bool = False) -> TuneReport:
    """``tpc_tune_batch``: choose (or load from the cache file) the launch
    choices of the pending batch; they are set on ``clusterers[0]``."""
    lib = load_library()
    arr = (ctypes.c_void_p * len(clusterers))(*[c.handle.value for c in clusterers])
    rep = TuneReport()
    _check(lib.tpc_tune_batch(arr, len(clusterers), None if cache_path is None else cache_path.encode(),
                              1 if force else 0, ctypes.byref(rep)), "tpc_tune_batch")
    return rep


def tune_cache_lookup(path: str, key: str):
    """(Tuning, ms) stored for key in the tuner's cache file, or None."""
    lib = load_library()
    t, ms = Tuning(), ctypes.c_double()
    rc = lib.tpc_tune_cache_lookup(path.encode(), key.encode(), ctypes.byref(t), ctypes.byref(ms))
    if rc == -10:   # TPC_ERR_STATE: no such file or key
        return None
    _check(rc, "tpc_tune_cache_lookup")
    return t, ms.value


def tune_cache_store(path: str, key: str, tuning: "Tuning | dict", ms: float):
    lib = load_library()
    if isinstance(tuning, dict):
        tuning = Tuning(**tuning)
    _check(lib.tpc_tune_cache_store(path.encode(), key.encode(), ctypes.byref(tuning), ms),
           "tpc_tune_cache_store")


class Filler:
    """Hit buffer filling (Algorithm 2), see ``tpc_filler_create``.  Host-side:
    ``store`` hits in arrival order, then ``take`` or ``send`` the buffers it
    has sent, oldest first."""

    def __init__(self, b: int, b_t: int, t: int, t_closing: int):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.tpc_filler_create(b, b_t, t, t_closing, ctypes.byref(h)), "tpc_filler_create")
        self._h, self._lib = h, lib

    def store(self, hits):
        a = np.ascontiguousarray(hits)
        if a.dtype != HIT_DTYPE:
            raise TypeError(f"hits must have dtype {HIT_DTYPE}")
        _check(self._lib.tpc_filler_store(self._h, a.ctypes.data if len(a) else None, len(a)),
               "tpc_filler_store")

    def finish(self):
        _check(self._lib.tpc_filler_finish(self._h), "tpc_filler_finish")

    def ready(self) -> tuple[int, int]:
        """(buffers waiting, hits in the oldest)."""
        nb, nh = ctypes.c_size_t(), ctypes.c_size_t()
        _check(self._lib.tpc_filler_ready(self._h, ctypes.byref(nb), ctypes.byref(nh)),
               "tpc_filler_ready")
        return nb.value, nh.value

    def take(self):
        """The oldest sent buffer as (hits, arrival indices, cut), or None."""
        nb, nh = self.ready()
        if not nb:
            return None
        hits = np.empty(nh, dtype=HIT_DTYPE)
        idx = np.empty(nh, dtype=np.uint64)
        n, cut = ctypes.c_size_t(), ctypes.c_uint64()
        _check(self._lib.tpc_filler_take(self._h, hits.ctypes.data, idx.ctypes.data, nh,
                                         ctypes.byref(n), ctypes.byref(cut)), "tpc_filler_take")
        return hits, idx, cut.value

    def take_into(self, hits, indices=None):
        """Take the oldest sent buffer into caller arrays (HIT_DTYPE records,
        uint64 indices or None); returns (n, cut), or None if none is waiting."""
        if hits.dtype != HIT_DTYPE or not hits.flags.c_contiguous:
            raise TypeError("hits must be a contiguous HIT_DTYPE array")
        if indices is not None and (indices.dtype != np.uint64 or len(indices) < len(hits)
                                    or not indices.flags.c_contiguous):
            raise TypeError("indices must be a contiguous uint64 array at least as long as hits")
        n, cut = ctypes.c_size_t(), ctypes.c_uint64()
        rc = self._lib.tpc_filler_take(self._h, hits.ctypes.data, None if indices is None else
                                       indices.ctypes.data, len(hits), ctypes.byref(n), ctypes.byref(cut))
        if rc == -10:    # TPC_ERR_STATE: no buffer waiting
            return None
        _check(rc, "tpc_filler_take")
        return n.value, cut.value

    def send(self, clusterer):
        """sendToDevice: push the oldest sent buffer into a Clusterer; returns
        (arrival indices, cut), or None if no buffer is waiting."""
        nb, nh = self.ready()
        if not nb:
            return None
        idx = np.empty(nh, dtype=np.uint64)
        n, cut = ctypes.c_size_t(), ctypes.c_uint64()
        _check(self._lib.tpc_filler_send(self._h, clusterer.handle, idx.ctypes.data, nh,
                                         ctypes.byref(n), ctypes.byref(cut)), "tpc_filler_send")
        return idx, cut.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tpc_filler_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class ServerResult(ctypes.Structure):
    """``tpc_server_result``."""
    _fields_ = [("tag", ctypes.c_uint64), ("stream", ctypes.c_int32), ("status", ctypes.c_int32),
                ("n_hits", ctypes.c_uint64), ("n_clusters", ctypes.c_uint64),
                ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    """``tpc_server_stats``."""
    _fields_ = [(name, ctypes.c_uint64) for name in
                ("budget", "in_use", "peak", "streams", "submitted", "admitted", "completed",
                 "failed", "rejected", "queued", "in_flight", "waits", "releases")]


class Server:
    """Serving loop (``tpc_server_*``): detector streams under one device-memory
    budget; chunks queue until memory and their stream are free.  Host
    buffers only: ``submit`` takes raw pointers (keep the memory alive until
    ``wait`` returns the chunk's result) or numpy arrays (kept alive here)."""

    def __init__(self, mem_budget: int):
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.tpc_server_create(mem_budget, ctypes.byref(h)), "tpc_server_create")
        self._h, self._lib = h, lib
        self._keep = {}

    def add_stream(self, width: int, height: int, dt: int, max_disorder: int) -> int:
        k = ctypes.c_int()
        _check(self._lib.tpc_server_add_stream(self._h, width, height, dt, max_disorder,
                                               ctypes.byref(k)), "tpc_server_add_stream")
        return k.value

    def submit_ptr(self, stream: int, hits_ptr, n: int, labels_ptr: int, indices_ptr, records_ptr: int,
                   cap: int, tag: int, end: bool = False):
        _check(self._lib.tpc_server_submit(self._h, stream, hits_ptr, n, labels_ptr, indices_ptr,
                                           records_ptr, cap, tag, int(end)), "tpc_server_submit")

    def submit(self, stream: int, hits, tag: int, cap: int | None = None, end: bool = False):
        """Queue numpy hits (or the end of the stream with hits=None); the
        result arrays are returned by ``wait`` as (result, labels, indices, records)."""
        a = None if hits is None else np.ascontiguousarray(hits)
        if a is not None and a.dtype != HIT_DTYPE:
            raise TypeError(f"hits must have dtype {HIT_DTYPE}")
        n = 0 if a is None else len(a)
        cap = cap if cap is not None else n + (1 << 20)
        lab = np.empty(cap, dtype=np.uint64)
        idx = np.empty(cap, dtype=np.uint64)
        rec = np.empty(cap, dtype=CLUSTER_DTYPE)
        self._keep[tag] = (a, lab, idx, rec)
        try:
            self.submit_ptr(stream, a.ctypes.data if n else None, n, lab.ctypes.data, idx.ctypes.data,
                            rec.ctypes.data, cap, tag, end)
        except Exception:
            self._keep.pop(tag, None)
            raise

    def wait_raw(self, timeout_s: float | None = None) -> ServerResult | None:
        """The next completed chunk's result record, or None on timeout."""
        r = ServerResult()
        us = -1 if timeout_s is None else int(timeout_s * 1e6)
        rc = self._lib.tpc_server_wait(self._h, ctypes.byref(r), us)
        if rc == -5:   # TPC_ERR_TIMEOUT
            return None
        _check(rc, "tpc_server_wait")
        return r

    def wait(self, timeout_s: float | None = None):
        """(result, labels, indices, records) of the next completed chunk
        submitted with ``submit``, or None on timeout."""
        r = self.wait_raw(timeout_s)
        if r is None:
            return None
        _, lab, idx, rec = self._keep.pop(r.tag)
        return r, lab[:r.n_hits], idx[:r.n_hits], rec[:r.n_clusters]

    def stats(self) -> dict:
        st = ServerStats()
        _check(self._lib.tpc_server_stats_get(self._h, ctypes.byref(st)), "tpc_server_stats_get")
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tpc_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
