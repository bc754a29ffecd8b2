"""The C-ABI library (no GPU needed): it builds, loads, and exports every
entry point include/tpc.h declares; the binding declares the same set; the
record layouts match on the C side."""
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tpc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tpc_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2412_11809_gb300 import build
    path = build.build()
    from paper_2412_11809_gb300 import binding
    return binding.load_library(path)


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "tpc_create" in names and "tpc_batch_flush" in names
    out = subprocess.run(["nm", "-D", "--defined-only",
                          os.path.join(ROOT, "paper_2412_11809_gb300", "_build", "libtpc.so")],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (tpc_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert getattr(lib, n) is not None


def test_binding_declares_header_set():
    from paper_2412_11809_gb300 import binding
    assert sorted(binding.SIGNATURES) == declared_functions()


def test_strerror_without_gpu(lib):
    assert lib.tpc_strerror(0) == b"ok"
    assert b"sensor" in lib.tpc_strerror(-2)
    assert lib.tpc_strerror(12345) == b"unknown status"


def test_checkpoint_argument_checks_without_gpu(lib):
    """Argument checks come before any CUDA call (no context needed)."""
    import ctypes
    n = ctypes.c_size_t()
    assert lib.tpc_snapshot(None, None, 0, ctypes.byref(n)) == -1
    assert lib.tpc_restore(None, None, 0) == -1
    buf = ctypes.create_string_buffer(64)
    assert lib.tpc_restore(None, buf, 64) == -1
    assert lib.tpc_forest(None, None, None, 0, ctypes.byref(n)) == -1
    assert lib.tpc_set_option(None, 5, 1) == -1


def test_record_layout_in_c():
    src = r'''
#include <stddef.h>
#include <stdio.h>
#include "tpc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(tpc_hit), offsetof(tpc_hit, toa),
         offsetof(tpc_hit, tot), sizeof(tpc_cluster), offsetof(tpc_cluster, first_toa),
         offsetof(tpc_cluster, cx));
  printf("%zu %zu %zu %zu %zu\n", sizeof(tpc_snapshot_header), offsetof(tpc_snapshot_header, dt),
         offsetof(tpc_snapshot_header, pushed), offsetof(tpc_snapshot_header, watermark),
         offsetof(tpc_snapshot_header, n_carry));
  return 0;
}'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe],
                       check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    from paper_2412_11809_gb300 import CLUSTER_DTYPE, HIT_DTYPE
    from paper_2412_11809_gb300.binding import SNAPSHOT_HEADER_DTYPE as S
    assert vals == [HIT_DTYPE.itemsize, HIT_DTYPE.fields["toa"][1], HIT_DTYPE.fields["tot"][1],
                    CLUSTER_DTYPE.itemsize, CLUSTER_DTYPE.fields["first_toa"][1],
                    CLUSTER_DTYPE.fields["cx"][1],
                    S.itemsize, S.fields["dt"][1], S.fields["pushed"][1],
                    S.fields["watermark"][1], S.fields["n_carry"][1]]


def test_product_path_does_not_import_oracle():
    """The CUDA path and the oracle share no code: nothing under the package
    imports, links or reads oracle/ (nor the CPU comparison baseline)."""
    pkg = os.path.join(ROOT, "paper_2412_11809_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower(), f
                assert "cpu_baseline" not in text and "tsplit" not in text, f


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: without the compiled library the binding raises."""
    from paper_2412_11809_gb300 import binding
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(RuntimeError):
            binding.load_library(str(tmp_path / "libtpc.so"))
    finally:
        binding._lib = saved
