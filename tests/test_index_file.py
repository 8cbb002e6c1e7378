"""The index file format of lnbnn_index_save / lnbnn_index_load: files built
here from the documented layout, and the checks load makes before it touches
the device (these run without a GPU)."""
import ctypes
import os
import struct

import numpy as np
import pytest

from paper_1112_0059_gb300 import build, lnbnn


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lnbnn.load_library()


def fnv1a64(data: bytes) -> int:
    h = 1469598103934665603
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def index_file(ref: np.ndarray, labels: np.ndarray, n_classes: int, magic=b"LNBNNIX1", version=1, dim=None,
               weight=0) -> bytes:
    dim = ref.shape[1] if dim is None else dim
    body = magic + struct.pack("<IIqiI", version, dim, len(ref), n_classes, weight)
    body += np.ascontiguousarray(ref, np.uint8).tobytes() + np.ascontiguousarray(labels, "<i4").tobytes()
    return body + struct.pack("<Q", fnv1a64(body))


def load_status(lib, path) -> int:
    h = ctypes.c_void_p()
    code = lib.lnbnn_index_load(os.fsencode(str(path)), None, ctypes.byref(h))
    assert not h.value or code == 0
    if h.value:
        lib.lnbnn_index_destroy(h)
    return code


def test_rejected_files(lib, tmp_path):
    rng = np.random.default_rng(0)
    ref = rng.integers(0, 256, size=(40, 128), dtype=np.uint8)
    labels = (np.arange(40) % 3).astype(np.int32)
    good = index_file(ref, labels, 3)
    assert load_status(lib, tmp_path / "missing.bin") == 12
    cases = {
        "empty": b"",
        "magic": index_file(ref, labels, 3, magic=b"LNBNNIX2"),
        "version": index_file(ref, labels, 3, version=2),
        "dim": index_file(ref, labels, 3, dim=64),
        "truncated": good[:-9],
        "trailing": good + b"\0",
        "hash": good[:100] + bytes([good[100] ^ 1]) + good[101:],  # one flipped descriptor bit
        # the row layout: 128 bytes without a location weight, 130 with one of at most 48
        "weight on 128-byte rows": index_file(ref, labels, 3, weight=5),
        "129-byte rows": index_file(np.zeros((40, 129), np.uint8), labels, 3),
        "location weight 49": index_file(np.zeros((40, 130), np.uint8), labels, 3, weight=49),
        "130 bytes declared, 128 stored": index_file(ref, labels, 3, dim=130, weight=2),
    }
    for name, data in cases.items():
        (tmp_path / name).write_bytes(data)
        assert load_status(lib, tmp_path / name) == 12, name
    h = ctypes.c_void_p()
    assert lib.lnbnn_index_load(None, None, ctypes.byref(h)) == 1
    assert lib.lnbnn_index_load(b"x", None, None) == 1
    assert lib.lnbnn_index_save(None, b"x") == 1


def test_intact_file_passes_the_checks(lib, tmp_path):
    """A file written from the documented layout passes every check; what
    follows needs the device (without one the status is a device error)."""
    rng = np.random.default_rng(1)
    ref = rng.integers(0, 256, size=(25, 128), dtype=np.uint8)
    (tmp_path / "ok").write_bytes(index_file(ref, np.zeros(25, np.int32), 1))
    torch = pytest.importorskip("torch")
    code = load_status(lib, tmp_path / "ok")
    if torch.cuda.is_available():
        assert code == 0
    else:
        assert code not in (0, 1, 12), code
