"""Python binding of the C ABI in include/lnbnn.h (argument marshalling only).

Every step of the classifier runs in the CUDA library ``_lib/liblnbnn.so``;
this module passes device pointers (from PyTorch CUDA tensors), sizes and the
current CUDA stream, and turns status codes into exceptions.  There is no CPU
fallback: without the built library every call raises.

Method: McCann & Lowe, "Local Naive Bayes Nearest Neighbor for Image
Classification" -- Alg. 1 (NBNN) and Alg. 2 (LocalNBNN).

``Index``        the merged reference index (128-byte rows, or 130-byte rows
                 with a location weight); ``knn_search``, ``lnbnn_classify``
                 (exact, or ``shortlist=m`` for the FP8 shortlist form),
                 ``nbnn_classify``, ``nbnn_logodds_classify`` (Section 3.1),
                 ``classify_host`` (host buffers), ``save`` / ``load``,
                 ``autotune`` / ``plan_splits`` / ``plan_search``, ``prepare_fp8``,
                 ``profile_enable`` / ``profile_read``, ``sync``
``Workspace``    device scratch of one in-flight call (allocation-free calls,
                 several streams, CUDA graph capture)
``knn_search_noalloc``, ``debug_fail_allocations``, ``LnbnnError``
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblnbnn.so")

STATUS = {
    0: "ok",
    1: "invalid argument",
    2: "label out of range",
    3: "a class has no reference descriptor",
    4: "k out of range",
    5: "device out of memory",
    6: "CUDA error",
    7: "device wait timed out",
    8: "unsupported device",
    9: "invalid image offsets",
    10: "problem larger than a workspace or the scratch of knn_search_noalloc",
    11: "the index has no FP8 operand (call prepare_fp8 first)",
    12: "file could not be written or read, or is not an intact index file",
}
MAX_K = 255

EXPORTS = ["lnbnn_index_create", "lnbnn_index_destroy", "lnbnn_index_info", "knn_search", "lnbnn_classify",
           "nbnn_classify", "lnbnn_classify_host", "nbnn_classify_host", "lnbnn_sync", "lnbnn_profile_enable",
           "lnbnn_profile_read", "lnbnn_status_string", "knn_search_noalloc", "lnbnn_workspace_create",
           "lnbnn_workspace_destroy", "knn_search_ws", "lnbnn_classify_ws", "nbnn_classify_ws",
           "lnbnn_index_prepare_fp8", "knn_search_fp8", "lnbnn_classify_fp8", "knn_search_fp8_ws",
           "lnbnn_classify_fp8_ws", "lnbnn_classify_fp8_host", "lnbnn_autotune", "lnbnn_plan_splits",
           "lnbnn_plan_search", "lnbnn_set_schedule",
           "lnbnn_debug_fail_allocations", "lnbnn_set_start_gate", "lnbnn_index_save", "lnbnn_index_load",
           "nbnn_logodds_classify", "nbnn_logodds_classify_ws", "lnbnn_index_create_located", "lnbnn_index_layout"]


class Profile(ctypes.Structure):
    """Mirror of ``lnbnn_profile`` (include/lnbnn.h)."""
    _fields_ = [("calls", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("search_launches", ctypes.c_int64), ("search_ms", ctypes.c_double), ("other_ms", ctypes.c_double),
                ("search_sm_clock_ghz", ctypes.c_double), ("search_cycles_per_tile", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Tuning(ctypes.Structure):
    """Mirror of ``lnbnn_tuning`` (include/lnbnn.h)."""
    _fields_ = [("tile_ms", ctypes.c_double), ("wave_ms", ctypes.c_double), ("list_ms", ctypes.c_double),
                ("max_rel_error", ctypes.c_double), ("runs", ctypes.c_int32), ("exact_query_tiles", ctypes.c_int32),
                ("entry_ms", ctypes.c_double), ("exact_persistent", ctypes.c_int32),
                ("coarse_query_tiles", ctypes.c_int32), ("coarse_persistent", ctypes.c_int32),
                ("form_runs", ctypes.c_int32), ("form_ms", ctypes.c_double * 8)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["form_ms"] = list(self.form_ms)
        return d


class SearchPlan(ctypes.Structure):
    """Mirror of ``lnbnn_search_plan`` (include/lnbnn.h)."""
    _fields_ = [("splits", ctypes.c_int32), ("lists_per_row", ctypes.c_int32), ("split_len", ctypes.c_int64),
                ("list_storage", ctypes.c_int32), ("list_capacity", ctypes.c_int32), ("tile_m", ctypes.c_int32),
                ("tile_n", ctypes.c_int32), ("persistent", ctypes.c_int32), ("bound_per_tile", ctypes.c_int32),
                ("chunked", ctypes.c_int32)]

    STORAGE = {0: "registers", 1: "shared memory", 2: "global-memory heap"}

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_}
        d["list_storage"] = self.STORAGE.get(self.list_storage, self.list_storage)
        return d


class Schedule(ctypes.Structure):
    """Mirror of ``lnbnn_schedule`` (include/lnbnn.h)."""
    _fields_ = [("splits", ctypes.c_int32), ("query_tiles", ctypes.c_int32), ("persistent", ctypes.c_int32),
                ("bound_per_tile", ctypes.c_int32)]


class LnbnnError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, 'unknown status')} (status {code})")
        self.code = code


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblnbnn.so and declare its signatures.  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None and path == LIB_PATH:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        lib = ctypes.CDLL(path)
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.lnbnn_index_create.argtypes = [P, P, I64, I32, P, ctypes.POINTER(P)]
        lib.lnbnn_index_destroy.argtypes = [P]
        lib.lnbnn_index_destroy.restype = None
        lib.lnbnn_index_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I32)]
        lib.knn_search.argtypes = [P, P, I64, I32, P, P, P]
        lib.lnbnn_classify.argtypes = [P, P, I64, P, I64, I32, P, P, P]
        lib.nbnn_classify.argtypes = [P, P, I64, P, I64, P, P, P]
        lib.lnbnn_classify_host.argtypes = [P, P, I64, P, I64, I32, P, P, P]
        lib.nbnn_classify_host.argtypes = [P, P, I64, P, I64, P, P, P]
        lib.lnbnn_sync.argtypes = [P, P]
        lib.lnbnn_profile_enable.argtypes = [P, ctypes.c_int]
        lib.lnbnn_profile_read.argtypes = [P, ctypes.POINTER(Profile)]
        lib.lnbnn_workspace_create.argtypes = [P, I64, I32, ctypes.POINTER(P)]
        lib.lnbnn_workspace_destroy.argtypes = [P]
        lib.lnbnn_workspace_destroy.restype = None
        lib.knn_search_ws.argtypes = [P, P, P, I64, I32, P, P, P]
        lib.lnbnn_classify_ws.argtypes = [P, P, P, I64, P, I64, I32, P, P, P]
        lib.nbnn_classify_ws.argtypes = [P, P, P, I64, P, I64, P, P, P]
        lib.lnbnn_index_prepare_fp8.argtypes = [P, P]
        lib.knn_search_fp8.argtypes = [P, P, I64, I32, I32, P, P, P]
        lib.lnbnn_classify_fp8.argtypes = [P, P, I64, P, I64, I32, I32, P, P, P]
        lib.knn_search_fp8_ws.argtypes = [P, P, P, I64, I32, I32, P, P, P]
        lib.lnbnn_classify_fp8_ws.argtypes = [P, P, P, I64, P, I64, I32, I32, P, P, P]
        lib.lnbnn_classify_fp8_host.argtypes = [P, P, I64, P, I64, I32, I32, P, P, P]
        lib.lnbnn_autotune.argtypes = [P, P, ctypes.POINTER(Tuning)]
        lib.lnbnn_plan_splits.argtypes = [P, I64, ctypes.POINTER(I32)]
        lib.lnbnn_plan_search.argtypes = [P, I64, I32, I32, ctypes.POINTER(SearchPlan)]
        lib.lnbnn_plan_search.restype = ctypes.c_int
        lib.lnbnn_set_schedule.argtypes = [P, ctypes.POINTER(Schedule)]
        lib.lnbnn_set_schedule.restype = ctypes.c_int
        lib.lnbnn_debug_fail_allocations.argtypes = [I32]
        lib.lnbnn_debug_fail_allocations.restype = None
        lib.lnbnn_set_start_gate.argtypes = [P, P]
        lib.lnbnn_set_start_gate.restype = ctypes.c_int
        lib.lnbnn_index_save.argtypes = [P, ctypes.c_char_p]
        lib.lnbnn_index_save.restype = ctypes.c_int
        lib.lnbnn_index_load.argtypes = [ctypes.c_char_p, P, ctypes.POINTER(P)]
        lib.lnbnn_index_load.restype = ctypes.c_int
        lib.nbnn_logodds_classify.argtypes = [P, P, I64, P, I64, ctypes.c_double, I32, P, P, P, P]
        lib.lnbnn_index_create_located.argtypes = [P, P, I64, I32, I32, P, ctypes.POINTER(P)]
        lib.lnbnn_index_layout.argtypes = [P, ctypes.POINTER(I32), ctypes.POINTER(I32)]
        lib.nbnn_logodds_classify_ws.argtypes = [P, P, P, I64, P, I64, ctypes.c_double, I32, P, P, P, P]
        lib.lnbnn_status_string.argtypes = [ctypes.c_int]
        lib.lnbnn_status_string.restype = ctypes.c_char_p
        for name in ("lnbnn_index_create", "lnbnn_index_info", "knn_search", "lnbnn_classify", "nbnn_classify",
                     "lnbnn_classify_host", "nbnn_classify_host", "lnbnn_sync", "lnbnn_profile_enable",
                     "lnbnn_profile_read", "lnbnn_workspace_create", "knn_search_ws", "lnbnn_classify_ws",
                     "nbnn_classify_ws", "lnbnn_index_prepare_fp8", "knn_search_fp8", "lnbnn_classify_fp8",
                     "knn_search_fp8_ws", "lnbnn_classify_fp8_ws", "lnbnn_classify_fp8_host", "lnbnn_autotune",
                     "lnbnn_plan_splits", "nbnn_logodds_classify", "nbnn_logodds_classify_ws",
                     "lnbnn_index_create_located", "lnbnn_index_layout"):
            getattr(lib, name).restype = ctypes.c_int
        if path == LIB_PATH:
            _lib = lib
        return lib


def _check(code: int, where: str) -> None:
    if code != 0:
        raise LnbnnError(code, where)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


class Index:
    """Merged reference index (Alg. 2's single search structure plus the class
    lookup), also serving original NBNN.  Owns device memory until ``close()``.

    ``ref`` is uint8 [N, 128], or [N, 130] with ``location_weight`` w: rows
    carry a location (x, y) after the 128 appearance bytes and distances add
    w times the squared location difference (lnbnn_index_create_located);
    queries then have 130-byte rows too."""

    def __init__(self, ref, labels, n_classes: int, stream=None, location_weight: int | None = None):
        import torch
        self._lib = load_library()
        if ref.dim() != 2 or ref.shape[1] not in (128, 130):
            raise ValueError("ref must be uint8 [N, 128] or [N, 130]")
        if (ref.shape[1] == 130) != (location_weight is not None):
            raise ValueError("130-byte rows go with a location_weight, 128-byte rows without")
        self.n_ref = int(ref.shape[0])
        self.n_classes = int(n_classes)
        self.row_bytes = int(ref.shape[1])
        self.location_weight = int(location_weight or 0)
        h = ctypes.c_void_p()
        args = (_dev(ref, torch.uint8, "ref"), _dev(labels, torch.int32, "labels"), self.n_ref, self.n_classes)
        if location_weight is None:
            _check(self._lib.lnbnn_index_create(*args, _stream_ptr(stream), ctypes.byref(h)), "lnbnn_index_create")
        else:
            _check(self._lib.lnbnn_index_create_located(*args, int(location_weight), _stream_ptr(stream),
                                                        ctypes.byref(h)), "lnbnn_index_create_located")
        self._h = h

    def _q(self, queries):
        """Device pointer of a uint8 [M, row_bytes] query tensor."""
        import torch
        if queries.dim() != 2 or queries.shape[1] != self.row_bytes:
            raise ValueError(f"queries must be uint8 [M, {self.row_bytes}] for this index")
        return _dev(queries, torch.uint8, "queries")

    @classmethod
    def load(cls, path: str, stream=None) -> "Index":
        """An index from a file written by ``save`` (checked before use)."""
        lib = load_library()
        h = ctypes.c_void_p()
        _check(lib.lnbnn_index_load(os.fsencode(path), _stream_ptr(stream), ctypes.byref(h)), "lnbnn_index_load")
        ix = cls.__new__(cls)
        ix._lib, ix._h = lib, h
        n_ref, n_cls = ctypes.c_int64(), ctypes.c_int32()
        _check(lib.lnbnn_index_info(h, ctypes.byref(n_ref), ctypes.byref(n_cls)), "lnbnn_index_info")
        ix.n_ref, ix.n_classes = int(n_ref.value), int(n_cls.value)
        rb, lw = ctypes.c_int32(), ctypes.c_int32()
        _check(lib.lnbnn_index_layout(h, ctypes.byref(rb), ctypes.byref(lw)), "lnbnn_index_layout")
        ix.row_bytes, ix.location_weight = int(rb.value), int(lw.value)
        return ix

    def save(self, path: str) -> None:
        """Write the index's references and labels to ``path`` (lnbnn_index_save)."""
        _check(self._lib.lnbnn_index_save(self.handle, os.fsencode(path)), "lnbnn_index_save")

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.lnbnn_index_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise ValueError("index is closed")
        return self._h

    def workspace(self, max_queries: int, max_k: int) -> "Workspace":
        """Device scratch for calls of at most max_queries descriptors and k <= max_k
        (no allocation inside those calls; one per concurrent stream)."""
        return Workspace(self, max_queries, max_k)

    def autotune(self, stream=None) -> dict:
        """Fit the split-N schedule model on the device (changes speed, never results)."""
        t = Tuning()
        _check(self._lib.lnbnn_autotune(self.handle, _stream_ptr(stream), ctypes.byref(t)), "lnbnn_autotune")
        return t.as_dict()

    def plan_splits(self, n_queries: int) -> int:
        """Reference splits a search of n_queries descriptors would use."""
        out = ctypes.c_int32()
        _check(self._lib.lnbnn_plan_splits(self.handle, int(n_queries), ctypes.byref(out)), "lnbnn_plan_splits")
        return out.value

    def plan_search(self, n_queries: int, k1: int, fp8: bool = False) -> dict:
        """How a search keeping the k1 nearest of n_queries descriptors would be
        launched (exact scan, or the FP8 coarse pass with k1 = shortlist)."""
        out = SearchPlan()
        _check(self._lib.lnbnn_plan_search(self.handle, int(n_queries), int(k1), int(bool(fp8)), ctypes.byref(out)),
               "lnbnn_plan_search")
        return out.as_dict()

    def set_schedule(self, splits: int = 0, query_tiles: int = 0, persistent: int = -1,
                     bound_per_tile: int = -1, automatic: bool = False) -> None:
        """Fix parts of the scans' launch schedule (0 / -1: automatic); speed
        only, never results.  ``automatic=True`` restores every choice."""
        sch = None if automatic else ctypes.byref(Schedule(splits, query_tiles, persistent, bound_per_tile))
        _check(self._lib.lnbnn_set_schedule(self.handle, sch), "lnbnn_set_schedule")

    def set_start_gate(self, gate=None) -> None:
        """Test hook: search kernels wait (at most 1 s) for the uint32/int32 device
        word ``gate`` to be nonzero; None removes the gate."""
        import torch
        ptr = None if gate is None else _dev(gate, gate.dtype, "gate")
        if gate is not None and gate.dtype not in (torch.int32,):
            raise TypeError("gate must be an int32 CUDA tensor")
        _check(self._lib.lnbnn_set_start_gate(self.handle, ptr), "lnbnn_set_start_gate")
        self._gate = gate  # keep the word alive while it is installed

    def prepare_fp8(self, stream=None) -> None:
        """Build the E4M3 operand of the FP8 shortlist search (once)."""
        _check(self._lib.lnbnn_index_prepare_fp8(self.handle, _stream_ptr(stream)), "lnbnn_index_prepare_fp8")

    def knn_search(self, queries, k: int, stream=None, workspace=None, out=None, shortlist: int | None = None):
        """NN(d, k): ``(idx int32 [M, k], dist int32 [M, k])`` by (distance, row); exact, or
        with ``shortlist`` the FP8 shortlist search (exact distances of the rows it finds)."""
        import torch
        m = int(queries.shape[0])
        idx, dist = out if out is not None else (
            torch.empty((m, k), dtype=torch.int32, device=queries.device),
            torch.empty((m, k), dtype=torch.int32, device=queries.device))
        q = self._q(queries)
        tail = (_dev(idx, torch.int32, "idx"), _dev(dist, torch.int32, "dist"), _stream_ptr(stream))
        if shortlist is None:
            if workspace is None:
                _check(self._lib.knn_search(self.handle, q, m, k, *tail), "knn_search")
            else:
                _check(self._lib.knn_search_ws(self.handle, workspace.handle, q, m, k, *tail), "knn_search_ws")
        elif workspace is None:
            _check(self._lib.knn_search_fp8(self.handle, q, m, k, int(shortlist), *tail), "knn_search_fp8")
        else:
            _check(self._lib.knn_search_fp8_ws(self.handle, workspace.handle, q, m, k, int(shortlist), *tail),
                   "knn_search_fp8_ws")
        return idx, dist

    def lnbnn_classify(self, queries, offsets, k: int, stream=None, out=None, workspace=None,
                       shortlist: int | None = None):
        """Alg. 2: ``(totals int64 [n_img, C], classes int32 [n_img])``; with ``shortlist``
        the neighbours come from the FP8 shortlist search."""
        import torch
        m, n_img = int(queries.shape[0]), int(offsets.shape[0]) - 1
        totals, classes = out if out is not None else (
            torch.empty((n_img, self.n_classes), dtype=torch.int64, device=queries.device),
            torch.empty((n_img,), dtype=torch.int32, device=queries.device))
        head = (self._q(queries), m, _dev(offsets, torch.int64, "offsets"), n_img, k)
        tail = (_dev(totals, torch.int64, "totals"), _dev(classes, torch.int32, "classes"), _stream_ptr(stream))
        if shortlist is None:
            if workspace is None:
                _check(self._lib.lnbnn_classify(self.handle, *head, *tail), "lnbnn_classify")
            else:
                _check(self._lib.lnbnn_classify_ws(self.handle, workspace.handle, *head, *tail), "lnbnn_classify_ws")
        elif workspace is None:
            _check(self._lib.lnbnn_classify_fp8(self.handle, *head, int(shortlist), *tail), "lnbnn_classify_fp8")
        else:
            _check(self._lib.lnbnn_classify_fp8_ws(self.handle, workspace.handle, *head, int(shortlist), *tail),
                   "lnbnn_classify_fp8_ws")
        return totals, classes

    def nbnn_classify(self, queries, offsets, stream=None, out=None, workspace=None):
        """Alg. 1: ``(totals int64 [n_img, C], classes int32 [n_img])``."""
        import torch
        m, n_img = int(queries.shape[0]), int(offsets.shape[0]) - 1
        totals, classes = out if out is not None else (
            torch.empty((n_img, self.n_classes), dtype=torch.int64, device=queries.device),
            torch.empty((n_img,), dtype=torch.int32, device=queries.device))
        args = (self._q(queries), m, _dev(offsets, torch.int64, "offsets"), n_img,
                _dev(totals, torch.int64, "totals"), _dev(classes, torch.int32, "classes"), _stream_ptr(stream))
        if workspace is None:
            _check(self._lib.nbnn_classify(self.handle, *args), "nbnn_classify")
        else:
            _check(self._lib.nbnn_classify_ws(self.handle, workspace.handle, *args), "nbnn_classify_ws")
        return totals, classes

    def nbnn_logodds_classify(self, queries, offsets, beta: float, positive_only: bool = False, stream=None,
                              out=None, workspace=None):
        """NBNN as a sum of log-odds increments (Section 3.1), posterior
        P(C|d) ~ exp(-beta ||d - NN_C(d)||^2); positive_only keeps only the
        increments > 0 (Table 1).  Returns ``(totals float64 [n_img, C],
        classes int32 [n_img], increments added int64 [n_img])``."""
        import torch
        m, n_img = int(queries.shape[0]), int(offsets.shape[0]) - 1
        totals, classes, counts = out if out is not None else (
            torch.empty((n_img, self.n_classes), dtype=torch.float64, device=queries.device),
            torch.empty((n_img,), dtype=torch.int32, device=queries.device),
            torch.empty((n_img,), dtype=torch.int64, device=queries.device))
        args = (self._q(queries), m, _dev(offsets, torch.int64, "offsets"), n_img,
                float(beta), int(bool(positive_only)), _dev(totals, torch.float64, "totals"),
                _dev(classes, torch.int32, "classes"), _dev(counts, torch.int64, "n_increments"),
                _stream_ptr(stream))
        if workspace is None:
            _check(self._lib.nbnn_logodds_classify(self.handle, *args), "nbnn_logodds_classify")
        else:
            _check(self._lib.nbnn_logodds_classify_ws(self.handle, workspace.handle, *args),
                   "nbnn_logodds_classify_ws")
        return totals, classes, counts

    def classify_host(self, queries: np.ndarray, offsets: np.ndarray, k: int | None, totals: np.ndarray | None = None,
                      classes: np.ndarray | None = None, stream=None, shortlist: int | None = None):
        """Host-buffer form (k=None -> original NBNN; shortlist -> FP8 shortlist
        search).  numpy in, numpy out; pinned host arrays give the fastest copies."""
        q = np.ascontiguousarray(queries, dtype=np.uint8)
        if q.ndim != 2 or q.shape[1] != self.row_bytes:
            raise ValueError(f"queries must be uint8 [M, {self.row_bytes}] for this index")
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        n_img = off.shape[0] - 1
        if totals is None:
            totals = np.empty((n_img, self.n_classes), dtype=np.int64)
        if classes is None:
            classes = np.empty((n_img,), dtype=np.int32)
        p = lambda a: ctypes.c_void_p(a.ctypes.data)
        if shortlist is not None:
            code = self._lib.lnbnn_classify_fp8_host(self.handle, p(q), q.shape[0], p(off), n_img, k, int(shortlist),
                                                     p(totals), p(classes), _stream_ptr(stream))
        elif k is None:
            code = self._lib.nbnn_classify_host(self.handle, p(q), q.shape[0], p(off), n_img, p(totals), p(classes),
                                                _stream_ptr(stream))
        else:
            code = self._lib.lnbnn_classify_host(self.handle, p(q), q.shape[0], p(off), n_img, k, p(totals),
                                                 p(classes), _stream_ptr(stream))
        _check(code, "classify_host")
        return totals, classes

    def profile_enable(self, enable: bool = True) -> None:
        """Start (and reset) or stop the per-call device-time profile."""
        _check(self._lib.lnbnn_profile_enable(self.handle, 1 if enable else 0), "lnbnn_profile_enable")

    def profile_read(self) -> dict:
        """Sums since the last enable: calls, kernel launches, search / other device ms."""
        p = Profile()
        _check(self._lib.lnbnn_profile_read(self.handle, ctypes.byref(p)), "lnbnn_profile_read")
        return p.as_dict()

    def sync(self, stream=None) -> None:
        """Wait for the stream and raise any device-side error (timeout, offsets)."""
        _check(self._lib.lnbnn_sync(self.handle, _stream_ptr(stream)), "lnbnn_sync")


class Workspace:
    """Device scratch of one in-flight call (see ``lnbnn_workspace_create``)."""

    def __init__(self, index: Index, max_queries: int, max_k: int):
        self._lib = index._lib
        self.index = index
        self.max_queries, self.max_k = int(max_queries), int(max_k)
        h = ctypes.c_void_p()
        _check(self._lib.lnbnn_workspace_create(index.handle, self.max_queries, self.max_k, ctypes.byref(h)),
               "lnbnn_workspace_create")
        self._h = h

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise ValueError("workspace is closed")
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.lnbnn_workspace_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def debug_fail_allocations(count: int) -> None:
    """Test hook: the library's next ``count`` device allocations fail (OOM)."""
    load_library().lnbnn_debug_fail_allocations(int(count))


def knn_search_noalloc(ref, queries, k: int, stream=None):
    """knn_search without an index and without any device allocation by the
    library: every intermediate lives in the library's fixed 64 MiB device
    scratch array.  For callers that must not allocate device memory (a host
    framework that owns all allocations, or code that cannot take the device
    synchronisation cudaMalloc/cudaFree imply).  Calls share that array, so
    calls that overlap on the GPU race.  The output tensors here are allocated
    by PyTorch, the caller; a caller with its own buffers passes them to the C
    entry point directly.  Returns ``(idx int32 [M, k], dist int32 [M, k])``."""
    import torch
    lib = load_library()
    if not hasattr(lib.knn_search_noalloc, "_declared"):
        P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
        lib.knn_search_noalloc.argtypes = [P, I64, P, I64, I32, P, P, P]
        lib.knn_search_noalloc.restype = ctypes.c_int
        lib.knn_search_noalloc._declared = True
    for name, t in (("ref", ref), ("queries", queries)):
        if not isinstance(t, torch.Tensor) or t.dim() != 2 or t.shape[1] != 128:
            raise ValueError(f"{name} must be a uint8 [N, 128] tensor")
    if ref.device != queries.device:
        raise ValueError("ref and queries must be on the same CUDA device")
    m = int(queries.shape[0])
    with torch.cuda.device(queries.device):
        idx = torch.empty((m, k), dtype=torch.int32, device=queries.device)
        dist = torch.empty((m, k), dtype=torch.int32, device=queries.device)
        _check(lib.knn_search_noalloc(_dev(ref, torch.uint8, "ref"), int(ref.shape[0]),
                                      _dev(queries, torch.uint8, "queries"), m, k, _dev(idx, torch.int32, "idx"),
                                      _dev(dist, torch.int32, "dist"), _stream_ptr(stream)), "knn_search_noalloc")
    return idx, dist
