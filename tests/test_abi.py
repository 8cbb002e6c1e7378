"""The C-ABI library builds, loads on a machine without a GPU, and exports
every entry point include/lnbnn.h declares.  No compute call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "lnbnn.h")).read()
    return re.findall(r"LNBNN_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)


@pytest.fixture(scope="module")
def lib():
    from paper_1112_0059_gb300 import build, lnbnn
    build.build()
    return lnbnn.load_library()


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for n in ("lnbnn_index_create", "lnbnn_index_destroy", "lnbnn_classify", "nbnn_classify", "knn_search",
              "lnbnn_status_string", "lnbnn_sync"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_binding_names_match_header():
    from paper_1112_0059_gb300 import lnbnn
    assert sorted(lnbnn.EXPORTS) == sorted(declared_entry_points())


def test_status_strings(lib):
    for code in range(13):
        assert lib.lnbnn_status_string(code) != b"unknown status"
    assert b"prepare_fp8" in lib.lnbnn_status_string(11)
    assert b"k out of range" in lib.lnbnn_status_string(4)


def test_argument_errors_need_no_gpu(lib):
    out = ctypes.c_void_p()
    # null reference pointer: rejected before any CUDA call
    assert lib.lnbnn_index_create(None, None, 10, 2, None, ctypes.byref(out)) == 1
    assert not out.value
    # calls on a null index are rejected
    assert lib.knn_search(None, None, 0, 1, None, None, None) == 1
    assert lib.lnbnn_classify(None, None, 0, None, 0, 1, None, None, None) == 1
    assert lib.nbnn_classify(None, None, 0, None, 0, None, None, None) == 1
    assert lib.lnbnn_sync(None, None) == 1
    assert lib.lnbnn_index_prepare_fp8(None, None) == 1
    assert lib.knn_search_fp8(None, None, 0, 1, 8, None, None, None) == 1
    assert lib.lnbnn_classify_fp8(None, None, 0, None, 0, 1, 8, None, None, None) == 1
    assert lib.lnbnn_classify_fp8(None, None, 0, None, 0, 1, 0, None, None, None) == 4  # shortlist 0: no FP8 call
    assert lib.lnbnn_classify_fp8_ws(None, None, None, 0, None, 0, 1, 8, None, None, None) == 1
    assert lib.lnbnn_set_start_gate(None, None) == 1
    lib.lnbnn_debug_fail_allocations(2)  # a process-wide counter: needs no device
    lib.lnbnn_debug_fail_allocations(0)
    lib.lnbnn_index_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_1112_0059_gb300 import lnbnn
    with pytest.raises(ImportError):
        lnbnn.load_library(str(tmp_path / "missing.so"))


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1112_0059_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "lnbnn_oracle" not in text, f


def test_noalloc_binding_checks_shapes_before_any_call(lib):
    # rows of 64 bytes would make the kernels read past the end of the buffers:
    # the binding refuses them before the C entry point is reached
    torch = pytest.importorskip("torch")
    from paper_1112_0059_gb300 import lnbnn
    good = torch.zeros((10, 128), dtype=torch.uint8)
    bad = torch.zeros((10, 64), dtype=torch.uint8)
    for ref, q in ((bad, good), (good, bad), (good.reshape(-1), good)):
        with pytest.raises(ValueError):
            lnbnn.knn_search_noalloc(ref, q, 3)
