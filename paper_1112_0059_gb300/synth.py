"""Seeded synthetic SIFT-like workloads for Local NBNN.

This module only draws random numbers and lays them out; it holds none of the
classifier's arithmetic.  Both the CUDA path and the CPU oracle consume the
bytes it produces, so parity never depends on how the generator is read.

Recipe (one reading of the workload description, applied to every size):

* A shared pool of 64 prototype vectors, each coordinate ~ U[0, 128).
* Class ``c`` picks 16 distinct pool entries and jitters each coordinate by
  N(0, 20^2): these are its 16 class prototypes.
* One descriptor of class ``c``: a uniformly chosen class prototype, plus
  N(0, 12^2) noise per coordinate, each coordinate then zeroed independently
  with probability 0.3, clipped to [0, 255] and rounded half-to-even to uint8.
* Reference images are laid out class by class (class 0's images first), so
  the merged reference set is class-sorted; label = class.
* Query image ``j`` belongs to class ``j mod C``.
* Locations (for location-weighted descriptors, 130-byte rows): every class
  prototype has a home position ~ U[32, 224)^2 on a 0..255 image grid; a
  descriptor's (x, y) is the home of the prototype it was drawn from plus
  N(0, 24^2) per axis, clipped to [0, 255] and rounded half-to-even.  Drawn
  from streams of their own, so the 128 appearance bytes do not change.

Every random stream is keyed by (seed, purpose, class, image), so class ``c``'s
reference descriptors are the same bytes whatever the number of classes in the
index, and generation can be split across threads without changing a byte.

The descriptors stand in for the dense multi-scale SIFT of Caltech-101/256 used
in the paper's experiments (Section 5); those datasets are not used here.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field
from functools import lru_cache

import numpy as np

D = 128
POOL_SIZE = 64
PROTOS_PER_CLASS = 16
POOL_MEAN_HIGH = 128.0
PROTO_JITTER_SD = 20.0
NOISE_SD = 12.0
ZERO_PROB = 0.3

# stream purposes
_POOL, _CLASS, _REF, _QUERY, _COUNTS, _LOC = 0, 1, 2, 3, 4, 5
LOC_HOME_LOW, LOC_HOME_HIGH = 32.0, 224.0
LOC_SD = 24.0


@dataclass(frozen=True)
class Workload:
    """A synthetic Local NBNN workload.

    ``query_counts`` is ``("fixed", n)``, ``("uniform", lo, hi)`` (inclusive
    integers) or ``("loguniform", lo, hi)``.
    """

    name: str
    n_classes: int
    ref_imgs_per_class: int
    ref_desc_per_img: int
    n_query_imgs: int
    query_counts: tuple
    ks: tuple = (10,)
    seed: int = 0
    notes: str = ""

    @property
    def n_ref(self) -> int:
        return self.n_classes * self.ref_imgs_per_class * self.ref_desc_per_img

    def with_classes(self, n_classes: int) -> "Workload":
        """Same generator, first ``n_classes`` classes only."""
        import dataclasses
        return dataclasses.replace(self, n_classes=n_classes,
                                   name=f"{self.name}-C{n_classes}")

    def with_query_imgs(self, n_query_imgs: int) -> "Workload":
        import dataclasses
        return dataclasses.replace(self, n_query_imgs=n_query_imgs)


WORKLOADS = {
    "tiny": Workload("tiny", 10, 5, 100, 20, ("fixed", 100), ks=(10,),
                     notes="10 classes x 5 ref images x 100 descriptors; 20 query images x 100"),
    "caltech101-like": Workload("caltech101-like", 101, 15, 1000, 200, ("fixed", 1000), ks=(1, 10, 50),
                                notes="101 classes x 15 ref images x 1,000; 200 query images x 1,000"),
    "caltech256-like": Workload("caltech256-like", 256, 30, 1500, 500, ("fixed", 1500),
                                ks=(1, 2, 5, 10, 20, 50, 100),
                                notes="256 classes x 30 ref images x 1,500 (11.52M refs); 500 query images x 1,500"),
    "batched-uneven": Workload("batched-uneven", 256, 30, 1500, 1024, ("uniform", 200, 3000), ks=(10,),
                               notes="256-class index; 1,024 query images with U{200..3000} descriptors"),
    "serving": Workload("serving", 256, 30, 1500, 1024, ("loguniform", 100, 4000), ks=(10,),
                        notes="256-class index; query images with log-uniform [100, 4000] descriptors"),
}


def _rng(*key: int) -> np.random.Generator:
    return np.random.default_rng([int(k) for k in key])


@lru_cache(maxsize=8)
def _pool(seed: int) -> np.ndarray:
    return _rng(seed, _POOL).uniform(0.0, POOL_MEAN_HIGH, size=(POOL_SIZE, D)).astype(np.float32)


@lru_cache(maxsize=4096)
def class_prototypes(seed: int, c: int) -> np.ndarray:
    """The 16 prototypes of class ``c`` (float32 [16, 128])."""
    rng = _rng(seed, _CLASS, c)
    sel = rng.choice(POOL_SIZE, size=PROTOS_PER_CLASS, replace=False)
    jitter = rng.standard_normal((PROTOS_PER_CLASS, D), dtype=np.float32) * np.float32(PROTO_JITTER_SD)
    return _pool(seed)[sel] + jitter


def _descriptors(protos: np.ndarray, n: int, rng: np.random.Generator, out: np.ndarray) -> None:
    pick = rng.integers(0, protos.shape[0], size=n)
    x = protos[pick]
    x += rng.standard_normal((n, D), dtype=np.float32) * np.float32(NOISE_SD)
    x[rng.random((n, D), dtype=np.float32) < np.float32(ZERO_PROB)] = 0.0
    np.clip(x, 0.0, 255.0, out=x)
    np.rint(x, out=x)
    out[...] = x.astype(np.uint8)


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def reference_set(w: Workload) -> tuple[np.ndarray, np.ndarray]:
    """Merged reference set: ``(ref uint8 [N, 128], labels int32 [N])``, class-sorted."""
    per_img = w.ref_desc_per_img
    n_img = w.n_classes * w.ref_imgs_per_class
    ref = np.empty((n_img * per_img, D), dtype=np.uint8)
    labels = np.repeat(np.arange(w.n_classes, dtype=np.int32), w.ref_imgs_per_class * per_img)

    def one(g: int) -> None:
        c, m = divmod(g, w.ref_imgs_per_class)
        _descriptors(class_prototypes(w.seed, c), per_img, _rng(w.seed, _REF, c, m),
                     ref[g * per_img:(g + 1) * per_img])

    with ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(one, range(n_img)))
    return ref, labels


def query_counts(w: Workload) -> np.ndarray:
    """Descriptor count of each query image (int64 [n_query_imgs])."""
    kind = w.query_counts[0]
    if kind == "fixed":
        return np.full(w.n_query_imgs, int(w.query_counts[1]), dtype=np.int64)
    rng = _rng(w.seed, _COUNTS)
    lo, hi = int(w.query_counts[1]), int(w.query_counts[2])
    if kind == "uniform":
        return rng.integers(lo, hi + 1, size=w.n_query_imgs).astype(np.int64)
    if kind == "loguniform":
        u = rng.uniform(np.log(lo), np.log(hi), size=w.n_query_imgs)
        return np.clip(np.rint(np.exp(u)), lo, hi).astype(np.int64)
    raise ValueError(f"unknown query count rule {kind!r}")


def query_set(w: Workload, counts: np.ndarray | None = None
              ) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Flattened query images.

    Returns ``(queries uint8 [M, 128], offsets int64 [n_img + 1], true_class int32 [n_img])``;
    image ``j`` owns rows ``offsets[j]:offsets[j+1]`` and belongs to class ``j mod C``.
    """
    if counts is None:
        counts = query_counts(w)
    counts = np.asarray(counts, dtype=np.int64)
    offsets = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    q = np.empty((int(offsets[-1]), D), dtype=np.uint8)
    cls = (np.arange(len(counts)) % w.n_classes).astype(np.int32)

    def one(j: int) -> None:
        _descriptors(class_prototypes(w.seed, int(cls[j])), int(counts[j]),
                     _rng(w.seed, _QUERY, j), q[offsets[j]:offsets[j + 1]])

    with ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(one, range(len(counts))))
    return q, offsets, cls


def query_image(w: Workload, j: int, n: int) -> np.ndarray:
    """Descriptors of query image ``j`` alone (the same bytes ``query_set`` gives it)."""
    out = np.empty((n, D), dtype=np.uint8)
    _descriptors(class_prototypes(w.seed, j % w.n_classes), n, _rng(w.seed, _QUERY, j), out)
    return out


@lru_cache(maxsize=4096)
def prototype_homes(seed: int, c: int) -> np.ndarray:
    """Home positions (float32 [16, 2]) of class ``c``'s prototypes."""
    return _rng(seed, _LOC, c).uniform(LOC_HOME_LOW, LOC_HOME_HIGH, size=(PROTOS_PER_CLASS, 2)).astype(np.float32)


def _locations(seed: int, c: int, pick_rng: np.random.Generator, n: int, rng: np.random.Generator) -> np.ndarray:
    # the first draw of a descriptor stream is its prototype pick (see _descriptors)
    pick = pick_rng.integers(0, PROTOS_PER_CLASS, size=n)
    xy = prototype_homes(seed, c)[pick] + rng.standard_normal((n, 2), dtype=np.float32) * np.float32(LOC_SD)
    return np.rint(np.clip(xy, 0.0, 255.0)).astype(np.uint8)


def reference_locations(w: Workload) -> np.ndarray:
    """(x, y) of every reference descriptor (uint8 [N, 2]), row-aligned with ``reference_set``."""
    per_img = w.ref_desc_per_img
    out = np.empty((w.n_classes * w.ref_imgs_per_class * per_img, 2), dtype=np.uint8)
    for g in range(w.n_classes * w.ref_imgs_per_class):
        c, m = divmod(g, w.ref_imgs_per_class)
        out[g * per_img:(g + 1) * per_img] = _locations(w.seed, c, _rng(w.seed, _REF, c, m), per_img,
                                                        _rng(w.seed, _LOC, 1, c, m))
    return out


def query_locations(w: Workload, counts: np.ndarray | None = None) -> np.ndarray:
    """(x, y) of every query descriptor (uint8 [M, 2]), row-aligned with ``query_set``."""
    counts = query_counts(w) if counts is None else np.asarray(counts, dtype=np.int64)
    out = np.empty((int(counts.sum()), 2), dtype=np.uint8)
    at = 0
    for j, n in enumerate(counts):
        out[at:at + n] = _locations(w.seed, j % w.n_classes, _rng(w.seed, _QUERY, j), int(n),
                                    _rng(w.seed, _LOC, 2, j))
        at += n
    return out


def located(desc: np.ndarray, loc: np.ndarray) -> np.ndarray:
    """130-byte rows: the 128 appearance bytes, then (x, y)."""
    return np.ascontiguousarray(np.concatenate([desc, loc], axis=1), dtype=np.uint8)


def workload(name: str) -> Workload:
    return WORKLOADS[name]
