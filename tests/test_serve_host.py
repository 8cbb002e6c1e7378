"""Host logic of the serving loop: admission, buckets, arrivals, statistics."""
import collections

import numpy as np
import pytest

from paper_1112_0059_gb300 import serve, synth


def req(rid, n, t=0.0):
    return serve.Request(rid, np.zeros((n, 128), np.uint8), t)


def test_take_batch_is_fifo_and_respects_capacity():
    pending = collections.deque(req(i, n) for i, n in enumerate([300, 500, 200, 900, 10]))
    b1 = serve.take_batch(pending, 1000, 10)
    assert [r.rid for r in b1] == [0, 1, 2]  # 1000 descriptors exactly
    b2 = serve.take_batch(pending, 1000, 10)
    assert [r.rid for r in b2] == [3, 4]
    assert not pending and serve.take_batch(pending, 1000, 10) == []


def test_take_batch_does_not_skip_ahead():
    # A small request behind one that does not fit waits: arrival order is kept.
    pending = collections.deque([req(0, 700), req(1, 400), req(2, 100)])
    assert [r.rid for r in serve.take_batch(pending, 1000, 10)] == [0]
    assert [r.rid for r in pending] == [1, 2]


def test_take_batch_image_cap_and_oversize():
    pending = collections.deque(req(i, 1) for i in range(7))
    assert len(serve.take_batch(pending, 1000, 3)) == 3
    with pytest.raises(ValueError):
        serve.take_batch(collections.deque([req(9, 1001)]), 1000, 3)


def test_graph_buckets():
    b = serve.graph_buckets(16384)
    assert b[0] == 128 and b[-1] == 16384 and b == sorted(set(b))
    assert all(x % 128 == 0 for x in b)
    # every query tile up to 4,096, then consecutive buckets at most ~25% (or one tile) apart
    assert [x for x in b if x <= 4096] == list(range(128, 4097, 128))
    assert all(y <= max(x + 128, 1.25 * x + 128) for x, y in zip(b, b[1:]))
    assert serve.bucket_of(1, b) == 128 and serve.bucket_of(128, b) == 128 and serve.bucket_of(129, b) == 256
    assert serve.bucket_of(16384, b) == 16384
    with pytest.raises(ValueError):
        serve.bucket_of(16385, b)
    assert serve.graph_buckets(1000)[-1] == 1000


def test_poisson_requests_shape_and_rate():
    w = synth.workload("serving").with_classes(4)
    rs = serve.poisson_requests(w, 500.0, 400, seed=3)
    t = np.array([r.arrival for r in rs])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    assert 0.8 / 500 < np.mean(np.diff(t)) < 1.2 / 500
    n = np.array([len(r.descriptors) for r in rs])
    assert n.min() >= 100 and n.max() <= 4000
    # log-uniform [100, 4000]: median near sqrt(100 * 4000) = 632
    assert 450 < np.median(n) < 850
    # the bytes are those of the workload's own query images
    assert np.array_equal(rs[5].descriptors, synth.query_image(w, 5, len(rs[5].descriptors)))


def test_latency_stats_and_in_flight():
    rs = [req(0, 10, 0.0), req(1, 20, 0.1), req(2, 30, 0.2)]
    for r, d in zip(rs, (0.05, 0.3, 0.4)):
        r.done = d
    log = [(0.0, 0.05, 1, 10), (0.1, 0.3, 1, 20), (0.2, 0.4, 1, 30)]
    s = serve.latency_stats(rs, log)
    assert s["images"] == 3 and abs(s["images_per_s"] - 3 / 0.4) < 1e-9
    assert abs(s["query_descriptors_per_s"] - 60 / 0.4) < 1e-9
    assert abs(s["p50_ms"] - 200.0) < 1e-6
    assert s["max_batches_in_flight"] == 2 and s["batches"] == 3
    # back-to-back batches (one ends when the next starts) do not overlap
    assert serve.max_in_flight([(0, 1, 1, 1), (1, 2, 1, 1)]) == 1
