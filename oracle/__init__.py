"""CPU oracle for Local NBNN and original NBNN -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does.

The arithmetic lives in ``lnbnn_oracle.c`` (plain C, int64 results), built on
first use with the host C compiler into ``oracle/_build/``.  Every function
here only marshals numpy arrays.

Functions (paper: McCann & Lowe, "Local Naive Bayes Nearest Neighbor"):
  sqdist_matrix  -- ||q_i - r_j||^2, the distance of Alg. 1 and Alg. 2
  knn            -- NN(d, kk) of Alg. 2, ordered by (distance, index)
  class_min      -- NN_C(d) of Alg. 1 for every class
  local_nbnn     -- Alg. 2 (LocalNBNN), per-image int64 totals + argmin
  local_nbnn_closed_form -- the same totals by sum_i min(0, NN_C - dist_B)
  nbnn           -- Alg. 1 (original NBNN), per-image int64 totals + argmin

Each of these also takes 130-byte rows (128 appearance bytes, then 2 location
bytes) with ``location_weight=w``: the distance adds w times the squared
location difference (the alpha location weighting fixed in Section 5).

Coarse-shortlist form (this project's approximate search, in the place of the
approximate kd-tree search of Section 5; exact neighbours on the shortlist):
  e4m3_round     -- nearest FP8 E4M3 value of integers, ties to even mantissa
  coarse_matrix  -- ||q'||^2 + ||r'||^2 - 2 q~.r~ with x' = x - 64, x~ = E4M3(x')
  knn_coarse     -- the m smallest coarse values, reranked by exact distance
  local_nbnn_coarse -- Alg. 2 on the reranked neighbours

NBNN as a sum of log-odds increments (Section 3.1, with the "positive
increments only" variant of Table 1) is float64 numpy in ``logodds.py``, on
top of ``class_min``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lnbnn_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liblnbnn_oracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {
    -1: "invalid argument",
    -2: "label out of range",
    -3: "k out of range (need 1 <= k and k + 1 <= N)",
    -4: "a class has no reference descriptors",
    -5: "invalid offsets",
    -6: "out of memory",
}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}: {ERRORS.get(code, 'unknown')}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, no arch-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cc = os.environ.get("CC", "gcc")
        subprocess.check_call([cc, "-O3", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Oracle:
    """ctypes view of one build of ``lnbnn_oracle.c``."""

    def __init__(self, lib_path: str):
        lib = ctypes.CDLL(lib_path)
        P = ctypes.c_void_p
        I64, I32, INT = ctypes.c_int64, ctypes.c_int32, ctypes.c_int
        lib.oracle_sqdist_matrix.argtypes = [P, I64, P, I64, P]
        lib.oracle_knn.argtypes = [P, I64, P, I64, I32, P, P, INT]
        lib.oracle_class_min.argtypes = [P, P, I64, I32, P, I64, P, INT]
        for f in (lib.oracle_lnbnn, lib.oracle_lnbnn_closed_form):
            f.argtypes = [P, P, I64, I32, P, P, I64, I32, P, P, INT]
        lib.oracle_nbnn.argtypes = [P, P, I64, I32, P, P, I64, P, P, INT]
        lib.oracle_e4m3_round.argtypes = [P, I64, P]
        lib.oracle_coarse_matrix.argtypes = [P, I64, P, I64, P]
        lib.oracle_knn_coarse.argtypes = [P, I64, P, I64, I32, I32, P, P, INT]
        lib.oracle_lnbnn_coarse.argtypes = [P, P, I64, I32, P, P, I64, I32, I32, P, P, INT]
        lib.oracle_sqdist_matrix_w.argtypes = [P, I64, P, I64, I32, I64, P]
        lib.oracle_knn_w.argtypes = [P, I64, P, I64, I32, I32, I64, P, P, INT]
        lib.oracle_class_min_w.argtypes = [P, P, I64, I32, P, I64, I32, I64, P, INT]
        for f in (lib.oracle_lnbnn_w, lib.oracle_lnbnn_closed_form_w):
            f.argtypes = [P, P, I64, I32, P, P, I64, I32, I32, I64, P, P, INT]
        lib.oracle_nbnn_w.argtypes = [P, P, I64, I32, P, P, I64, I32, I64, P, P, INT]
        for f in (lib.oracle_sqdist_matrix, lib.oracle_knn, lib.oracle_class_min,
                  lib.oracle_lnbnn, lib.oracle_lnbnn_closed_form, lib.oracle_nbnn, lib.oracle_e4m3_round,
                  lib.oracle_coarse_matrix, lib.oracle_knn_coarse, lib.oracle_lnbnn_coarse,
                  lib.oracle_sqdist_matrix_w, lib.oracle_knn_w, lib.oracle_class_min_w, lib.oracle_lnbnn_w,
                  lib.oracle_lnbnn_closed_form_w, lib.oracle_nbnn_w):
            f.restype = ctypes.c_int
        self.lib = lib

    def sqdist_matrix(self, ref, q, location_weight=None) -> np.ndarray:
        """int64 [M, N] with entry (i, j) = ||q_i - r_j||^2 (location-weighted for 130-byte rows)."""
        ref, q, stride, w = _rows(ref, q, location_weight)
        out = np.empty((q.shape[0], ref.shape[0]), dtype=np.int64)
        _check(self.lib.oracle_sqdist_matrix_w(_p(ref), ref.shape[0], _p(q), q.shape[0], stride, w, _p(out)))
        return out

    def knn(self, ref, q, kk: int, threads: int = 0, location_weight=None) -> tuple[np.ndarray, np.ndarray]:
        """``(dist int64 [M, kk], idx int64 [M, kk])``: the kk nearest by (distance, index)."""
        ref, q, stride, w = _rows(ref, q, location_weight)
        dist = np.empty((q.shape[0], kk), dtype=np.int64)
        idx = np.empty((q.shape[0], kk), dtype=np.int64)
        _check(self.lib.oracle_knn_w(_p(ref), ref.shape[0], _p(q), q.shape[0], kk, stride, w, _p(dist),
                                     _p(idx), threads))
        return dist, idx

    def class_min(self, ref, labels, n_classes: int, q, threads: int = 0, location_weight=None) -> np.ndarray:
        """int64 [M, C]: NN_C(q_i); int64 max where class C has no reference."""
        ref, q, stride, w = _rows(ref, q, location_weight)
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        out = np.empty((q.shape[0], n_classes), dtype=np.int64)
        _check(self.lib.oracle_class_min_w(_p(ref), _p(labels), ref.shape[0], n_classes, _p(q),
                                           q.shape[0], stride, w, _p(out), threads))
        return out

    def _classify(self, fn, ref, labels, n_classes, q, offsets, k, threads, location_weight):
        ref, q, stride, w = _rows(ref, q, location_weight)
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        n_img = offsets.shape[0] - 1
        if n_img < 0 or offsets[-1] != q.shape[0]:
            raise OracleError(-5)
        totals = np.empty((n_img, n_classes), dtype=np.int64)
        classes = np.empty(n_img, dtype=np.int32)
        if k is None:
            code = fn(_p(ref), _p(labels), ref.shape[0], n_classes, _p(q), _p(offsets), n_img,
                      stride, w, _p(totals), _p(classes), threads)
        else:
            code = fn(_p(ref), _p(labels), ref.shape[0], n_classes, _p(q), _p(offsets), n_img, k,
                      stride, w, _p(totals), _p(classes), threads)
        _check(code)
        return totals, classes

    def local_nbnn(self, ref, labels, n_classes, q, offsets, k, threads: int = 0, location_weight=None):
        """Alg. 2: ``(totals int64 [n_img, C], classes int32 [n_img])``."""
        return self._classify(self.lib.oracle_lnbnn_w, ref, labels, n_classes, q, offsets, k, threads,
                              location_weight)

    def local_nbnn_closed_form(self, ref, labels, n_classes, q, offsets, k, threads: int = 0,
                               location_weight=None):
        """Local NBNN totals as sum_i min(0, NN_C(d_i) - dist_B(d_i)); small inputs."""
        return self._classify(self.lib.oracle_lnbnn_closed_form_w, ref, labels, n_classes, q,
                              offsets, k, threads, location_weight)

    def nbnn(self, ref, labels, n_classes, q, offsets, threads: int = 0, location_weight=None):
        """Alg. 1: ``(totals int64 [n_img, C], classes int32 [n_img])``."""
        return self._classify(self.lib.oracle_nbnn_w, ref, labels, n_classes, q, offsets, None,
                              threads, location_weight)

    def e4m3_round(self, x) -> np.ndarray:
        """Nearest FP8 E4M3 value of each integer (|x| <= 448), ties to even mantissa."""
        x = np.ascontiguousarray(x, dtype=np.int32)
        out = np.empty_like(x)
        _check(self.lib.oracle_e4m3_round(_p(x), x.size, _p(out)))
        return out

    def coarse_matrix(self, ref, q) -> np.ndarray:
        """int64 [M, N]: coarse(q_i, r_j) = ||q'||^2 + ||r'||^2 - 2 q~.r~."""
        ref, q = _u8(ref), _u8(q)
        out = np.empty((q.shape[0], ref.shape[0]), dtype=np.int64)
        _check(self.lib.oracle_coarse_matrix(_p(ref), ref.shape[0], _p(q), q.shape[0], _p(out)))
        return out

    def knn_coarse(self, ref, q, kk: int, m: int, threads: int = 0) -> tuple[np.ndarray, np.ndarray]:
        """``(dist, idx)`` int64 [M, kk]: exact rerank of the coarse shortlist of m."""
        ref, q = _u8(ref), _u8(q)
        dist = np.empty((q.shape[0], kk), dtype=np.int64)
        idx = np.empty((q.shape[0], kk), dtype=np.int64)
        _check(self.lib.oracle_knn_coarse(_p(ref), ref.shape[0], _p(q), q.shape[0], kk, m, _p(dist), _p(idx),
                                          threads))
        return dist, idx

    def local_nbnn_coarse(self, ref, labels, n_classes, q, offsets, k, m, threads: int = 0):
        """Alg. 2 on the neighbours of the coarse shortlist of m (m >= k + 1)."""
        ref, q = _u8(ref), _u8(q)
        labels = np.ascontiguousarray(labels, dtype=np.int32)
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        n_img = offsets.shape[0] - 1
        if n_img < 0 or offsets[-1] != q.shape[0]:
            raise OracleError(-5)
        totals = np.empty((n_img, n_classes), dtype=np.int64)
        classes = np.empty(n_img, dtype=np.int32)
        _check(self.lib.oracle_lnbnn_coarse(_p(ref), _p(labels), ref.shape[0], n_classes, _p(q), _p(offsets),
                                            n_img, k, m, _p(totals), _p(classes), threads))
        return totals, classes


def _u8(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.uint8)
    if a.ndim != 2 or a.shape[1] != 128:
        raise ValueError("descriptors must be uint8 [n, 128]")
    return a


def _rows(ref, q, location_weight):
    """Reference and query rows of one layout (128 bytes, or 130 with a
    location weight), their stride and the weight."""
    ref = np.ascontiguousarray(ref, dtype=np.uint8)
    q = np.ascontiguousarray(q, dtype=np.uint8)
    if ref.ndim != 2 or q.ndim != 2 or ref.shape[1] != q.shape[1] or ref.shape[1] not in (128, 130):
        raise ValueError("descriptors must be uint8 [n, 128] or [n, 130], the same for references and queries")
    if ref.shape[1] == 130:
        if location_weight is None or int(location_weight) < 0:
            raise ValueError("130-byte rows need a location weight >= 0")
        return ref, q, 130, int(location_weight)
    if location_weight not in (None, 0):
        raise ValueError("a location weight needs 130-byte rows")
    return ref, q, 128, 0


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(code: int) -> None:
    if code != 0:
        raise OracleError(code)


def compile_source(src: str, out_path: str) -> str:
    """Compile C source text ``src`` into a shared library at ``out_path``."""
    cc = os.environ.get("CC", "gcc")
    tmp = out_path + f".tmp{os.getpid()}"
    subprocess.run([cc, "-O3", "-std=c11", "-fPIC", "-shared", "-pthread", "-x", "c",
                    "-o", tmp, "-"], input=src.encode(), check=True)
    os.replace(tmp, out_path)
    return out_path


def source() -> str:
    with open(_SRC) as f:
        return f.read()


def default() -> Oracle:
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(build())
    return _lib


def sqdist_matrix(ref, q, location_weight=None):
    return default().sqdist_matrix(ref, q, location_weight)


def knn(ref, q, kk, threads=0, location_weight=None):
    return default().knn(ref, q, kk, threads, location_weight)


def class_min(ref, labels, n_classes, q, threads=0, location_weight=None):
    return default().class_min(ref, labels, n_classes, q, threads, location_weight)


def local_nbnn(ref, labels, n_classes, q, offsets, k, threads=0, location_weight=None):
    return default().local_nbnn(ref, labels, n_classes, q, offsets, k, threads, location_weight)


def local_nbnn_closed_form(ref, labels, n_classes, q, offsets, k, threads=0, location_weight=None):
    return default().local_nbnn_closed_form(ref, labels, n_classes, q, offsets, k, threads, location_weight)


def nbnn(ref, labels, n_classes, q, offsets, threads=0, location_weight=None):
    return default().nbnn(ref, labels, n_classes, q, offsets, threads, location_weight)


def e4m3_round(x):
    return default().e4m3_round(x)


def coarse_matrix(ref, q):
    return default().coarse_matrix(ref, q)


def knn_coarse(ref, q, kk, m, threads=0):
    return default().knn_coarse(ref, q, kk, m, threads)


def local_nbnn_coarse(ref, labels, n_classes, q, offsets, k, m, threads=0):
    return default().local_nbnn_coarse(ref, labels, n_classes, q, offsets, k, m, threads)


def host_threads() -> int:
    return os.cpu_count() or 1
