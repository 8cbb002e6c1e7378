"""Seeded generator determinism and the stored oracle answers on the tiny workload."""
import hashlib
import json
import os

import numpy as np

import oracle
from paper_1112_0059_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tiny_oracle.json")


def _h(a):
    return hashlib.sha256(a.tobytes()).hexdigest()


def test_tiny_inputs_match_golden_digests():
    g = json.load(open(GOLDEN))
    w = synth.workload("tiny")
    ref, labels = synth.reference_set(w)
    q, offsets, _ = synth.query_set(w)
    assert _h(ref) == g["sha256"]["ref"]
    assert _h(labels) == g["sha256"]["labels"]
    assert _h(q) == g["sha256"]["queries"]
    assert _h(offsets) == g["sha256"]["offsets"]


def test_tiny_oracle_matches_golden():
    g = json.load(open(GOLDEN))
    w = synth.workload("tiny")
    ref, labels = synth.reference_set(w)
    q, offsets, _ = synth.query_set(w)
    lt, lc = oracle.local_nbnn(ref, labels, w.n_classes, q, offsets, g["k"])
    nt, nc = oracle.nbnn(ref, labels, w.n_classes, q, offsets)
    assert lt.tolist() == g["local_nbnn"]["totals"] and lc.tolist() == g["local_nbnn"]["classes"]
    assert nt.tolist() == g["nbnn"]["totals"] and nc.tolist() == g["nbnn"]["classes"]
    d, j = oracle.knn(ref, q[:8], g["k"] + 1)
    assert d.tolist() == g["knn_first_8_rows"]["dist"] and j.tolist() == g["knn_first_8_rows"]["idx"]


def test_class_subset_is_prefix():
    w = synth.workload("tiny")
    full, lf = synth.reference_set(w)
    sub, ls = synth.reference_set(w.with_classes(4))
    assert np.array_equal(sub, full[:len(sub)]) and np.array_equal(ls, lf[:len(ls)])


def test_query_image_alone_matches_flattened():
    w = synth.workload("tiny")
    q, off, cls = synth.query_set(w)
    assert np.array_equal(synth.query_image(w, 7, 100), q[off[7]:off[8]])
    assert cls.tolist() == [j % 10 for j in range(20)]


def test_uneven_counts_in_range():
    w = synth.workload("batched-uneven")
    c = synth.query_counts(w)
    assert len(c) == 1024 and c.min() >= 200 and c.max() <= 3000
    s = synth.query_counts(synth.workload("serving"))
    assert s.min() >= 100 and s.max() <= 4000


def test_descriptor_statistics():
    w = synth.workload("tiny")
    ref, labels = synth.reference_set(w)
    assert ref.dtype == np.uint8 and ref.shape == (5000, 128)
    zero_frac = float((ref == 0).mean())
    assert 0.28 < zero_frac < 0.40  # 30% zeroed plus clipping at 0
    assert np.array_equal(labels, np.repeat(np.arange(10), 500))
