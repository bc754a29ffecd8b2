"""GB300 (sm_103a) clustering of Timepix hits into connected components.

The compute lives in the CUDA library ``_build/libtpc.so`` (C ABI in
``include/tpc.h``); this package is its binding.  See ``Clusterer``, the
serving loop ``Server`` and, for the host-side hit buffer filling of
Algorithm 2, ``Filler``.
"""
from .binding import (CLUSTER_DTYPE, HIT_DTYPE, Clusterer, Filler, Server, TpcError, Tuning,
                      batch_flush, load_library, tune_batch)

__all__ = ["CLUSTER_DTYPE", "HIT_DTYPE", "Clusterer", "Filler", "Server", "TpcError", "Tuning",
           "batch_flush", "load_library", "tune_batch"]
