"""tpc_cluster_static — the entry point that allocates nothing.

Some callers cannot call cudaMalloc (code running inside a CUDA-graph stream
capture, real-time readout loops that must not block on the allocator).
This test calls the entry point through the C ABI twice in a row on the
same inputs and checks both results against the regular context path
(tpc_push + tpc_flush + tpc_labels / tpc_cluster_features): labels exact,
integer features exact, centroids within 1e-5 relative.  It lives in a file
of its own that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2412_11809_gb300 import CLUSTER_DTYPE, Clusterer, binding  # noqa: E402

MAX_HITS = 65536


def _reference(hits, w, h, dt):
    with Clusterer(w, h, dt) as c:
        c.push(hits)
        c.flush()
        return c.labels(), c.features()


@pytest.mark.parametrize("sensor", ["256x256", "448x512"])
def test_static_entry_matches_context_path_twice(sensor):
    lib = binding.load_library()
    if sensor == "256x256":
        w, h = 256, 256
        hits, _ = synth.cfg1(scale=60000 / (64 * 2**20), seed=31)   # 60000 hits: 15 tiles, ragged tail
    else:   # larger than the shared-memory pixel table: linked band by band
        w, h = 448, 512
        hits, _ = synth.cfg4(scale=60000 / (512 * 2**20), seed=32)
    n = len(hits)
    assert 4096 * 14 < n <= MAX_HITS
    want_lab, want_rec = _reference(hits, w, h, 128)

    d_hits = torch.from_numpy(hits.view(np.uint8).reshape(-1, 16)).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):
        d_lab = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        d_rec = torch.zeros((n, CLUSTER_DTYPE.itemsize), dtype=torch.uint8, device="cuda")
        d_cnt = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        rc = lib.tpc_cluster_static(d_hits.data_ptr(), n, w, h, 128, d_lab.data_ptr(),
                                    d_rec.data_ptr(), n, d_cnt.data_ptr(),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, binding.STATUS.get(rc, rc)
        torch.cuda.synchronize()
        n_clusters, err = (int(v) for v in d_cnt.cpu().numpy())
        assert err == 0, f"call {call}: device error bits {err}"
        assert n_clusters == len(want_rec)
        lab = d_lab.cpu().numpy().view(np.uint64)
        np.testing.assert_array_equal(lab, want_lab, err_msg=f"call {call}")
        rec = d_rec.cpu().numpy().view(CLUSTER_DTYPE).reshape(-1)[:n_clusters]
        for k in ("label", "size", "sum_tot", "first_toa"):
            np.testing.assert_array_equal(rec[k], want_rec[k], err_msg=f"call {call} {k}")
        for k in ("cx", "cy"):
            np.testing.assert_allclose(rec[k], want_rec[k], rtol=1e-5, atol=0,
                                       err_msg=f"call {call} {k}")


def test_static_entry_rejects_oversize_batch():
    lib = binding.load_library()
    d_cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    rc = lib.tpc_cluster_static(None, MAX_HITS + 1, 256, 256, 128, None, None, 0,
                                d_cnt.data_ptr(), None)
    assert binding.STATUS[rc] == "TPC_ERR_ARG"
