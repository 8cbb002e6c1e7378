"""Serving loop: requests admitted while others run, batched together, give
each image the result it gets alone, equal to the oracle."""
import dataclasses

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lnbnn():
    from paper_1112_0059_gb300 import build, lnbnn
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    lnbnn.load_library()
    return lnbnn


@pytest.fixture(scope="module")
def setup(lnbnn):
    from paper_1112_0059_gb300 import serve, synth
    # The serving rule (log-uniform [100, 4000] descriptors per image) over a
    # small 6-class index, so that the oracle finishes in seconds.
    w = dataclasses.replace(synth.workload("serving"), n_classes=6, ref_imgs_per_class=4, ref_desc_per_img=500)
    ref, labels = synth.reference_set(w)
    reqs = serve.poisson_requests(w, 1e6, 24, seed=1)  # all but at once: batches form
    q = np.concatenate([r.descriptors for r in reqs])
    off = np.concatenate([[0], np.cumsum([len(r.descriptors) for r in reqs])]).astype(np.int64)
    ix = lnbnn.Index(torch.from_numpy(ref).cuda(), torch.from_numpy(labels).cuda(), w.n_classes)
    yield w, ref, labels, reqs, q, off, ix
    ix.close()


@pytest.mark.parametrize("method,graphs,shortlist", [("local", False, None), ("local", True, None),
                                                     ("nbnn", False, None), ("local", True, 32)])
def test_served_equals_alone_and_oracle(setup, method, graphs, shortlist):
    from paper_1112_0059_gb300 import serve
    w, ref, labels, reqs, q, off, ix = setup
    reqs = [dataclasses.replace(r, totals=None, cls=None, done=None, batch=None) for r in reqs]
    if shortlist:
        ix.prepare_fp8()
    with serve.Server(ix, k=10, method=method, slots=3, max_batch_queries=6144, max_batch_images=8,
                      graphs=graphs, shortlist=shortlist) as srv:
        done = srv.run(reqs)
        log = srv.log
    assert len(done) == len(reqs)
    stats = serve.latency_stats(done, log)
    # continuous batching happened: several images per batch, several batches in flight
    assert stats["mean_images_per_batch"] > 1.0
    assert stats["max_batches_in_flight"] >= 2
    if shortlist:
        ot, oc = oracle.local_nbnn_coarse(ref, labels, w.n_classes, q, off, 10, shortlist)
    elif method == "local":
        ot, oc = oracle.local_nbnn(ref, labels, w.n_classes, q, off, 10)
    else:
        ot, oc = oracle.nbnn(ref, labels, w.n_classes, q, off)
    by_id = {r.rid: r for r in done}
    for i, r in enumerate(reqs):
        got = by_id[r.rid]
        assert np.array_equal(got.totals, ot[i]) and got.cls == oc[i], f"image {i} (batch {got.batch})"
    # each image alone, through the plain call
    for i in range(0, len(reqs), 5):
        qd = torch.from_numpy(reqs[i].descriptors).cuda()
        od = torch.tensor([0, len(reqs[i].descriptors)], dtype=torch.int64, device="cuda")
        t, c = ix.lnbnn_classify(qd, od, 10, shortlist=shortlist) if method == "local" else ix.nbnn_classify(qd, od)
        ix.sync()
        assert np.array_equal(t.cpu().numpy()[0], by_id[reqs[i].rid].totals) and int(c[0]) == by_id[reqs[i].rid].cls


def test_rejects_request_larger_than_a_slot(setup):
    from paper_1112_0059_gb300 import serve
    w, ref, labels, reqs, q, off, ix = setup
    big = serve.Request(0, np.zeros((5000, 128), np.uint8), 0.0)
    with serve.Server(ix, k=10, slots=1, max_batch_queries=4096) as srv:
        with pytest.raises(ValueError):
            srv.run([big])


def test_serves_location_weighted_rows(lnbnn):
    """A location-weighted index (130-byte rows) behind the server: batched,
    graph-captured service gives every image the oracle's answer."""
    from paper_1112_0059_gb300 import serve, synth
    w = dataclasses.replace(synth.workload("serving"), n_classes=5, ref_imgs_per_class=3, ref_desc_per_img=400)
    ref, labels = synth.reference_set(w)
    ref = synth.located(ref, synth.reference_locations(w))
    plain = serve.poisson_requests(w, 1e6, 12, seed=3)
    rng = np.random.default_rng(4)
    reqs = [dataclasses.replace(r, descriptors=synth.located(
        r.descriptors, rng.integers(0, 256, size=(len(r.descriptors), 2)).astype(np.uint8))) for r in plain]
    q = np.concatenate([r.descriptors for r in reqs])
    off = np.concatenate([[0], np.cumsum([len(r.descriptors) for r in reqs])]).astype(np.int64)
    with lnbnn.Index(torch.from_numpy(ref).cuda(), torch.from_numpy(labels).cuda(), w.n_classes,
                     location_weight=6) as ix:
        with serve.Server(ix, k=10, slots=2, max_batch_queries=6144, max_batch_images=6, graphs=True) as srv:
            done = srv.run(reqs)
    ot, oc = oracle.local_nbnn(ref, labels, w.n_classes, q, off, 10, location_weight=6)
    by_id = {r.rid: r for r in done}
    for i, r in enumerate(reqs):
        assert np.array_equal(by_id[r.rid].totals, ot[i]) and by_id[r.rid].cls == oc[i], i
