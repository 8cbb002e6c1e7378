"""Location-weighted descriptors (130-byte rows: appearance, then (x, y); the
distance adds w times the squared location difference) on the GPU against the
oracle: bit-exact neighbours, distances, Local NBNN and NBNN totals and
classes, including the extreme values that bound the exactness argument."""
import dataclasses

import numpy as np
import pytest

import oracle
import oracle.logodds

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lnbnn():
    from paper_1112_0059_gb300 import build, lnbnn
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    lnbnn.load_library()
    return lnbnn


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def located_case(seed, N, M, C, hi=256, loc_hi=256):
    rng = np.random.default_rng(seed)
    ref = rng.integers(0, hi, size=(N, 130)).astype(np.uint8)
    q = rng.integers(0, hi, size=(M, 130)).astype(np.uint8)
    ref[:, 128:] = rng.integers(0, loc_hi, size=(N, 2))
    q[:, 128:] = rng.integers(0, loc_hi, size=(M, 2))
    labels = rng.integers(0, C, size=N).astype(np.int32)
    labels[:C] = np.arange(C)
    return ref, labels, q


@pytest.mark.parametrize("w", [0, 1, 7, 48])
def test_matches_oracle(lnbnn, w):
    # ragged: N not a multiple of 256, M = 301 not a multiple of 128
    ref, labels, q = located_case(100 + w, 5037, 301, 6)
    off = np.array([0, 100, 100, 301], np.int64)
    with lnbnn.Index(dev(ref), dev(labels), 6, location_weight=w) as ix:
        assert (ix.row_bytes, ix.location_weight) == (130, w)
        for k in (1, 10):
            idx, dist = ix.knn_search(dev(q), k)
            ix.sync()
            od, oj = oracle.knn(ref, q, k, location_weight=w)
            assert np.array_equal(idx.cpu().numpy(), oj) and np.array_equal(dist.cpu().numpy(), od), k
        t, c = ix.lnbnn_classify(dev(q), dev(off), 5)
        tn, cn = ix.nbnn_classify(dev(q), dev(off))
        ix.sync()
    ot, oc = oracle.local_nbnn(ref, labels, 6, q, off, 5, location_weight=w)
    assert np.array_equal(t.cpu().numpy(), ot) and np.array_equal(c.cpu().numpy(), oc)
    nt, nc = oracle.nbnn(ref, labels, 6, q, off, location_weight=w)
    assert np.array_equal(tn.cpu().numpy(), nt) and np.array_equal(cn.cpu().numpy(), nc)


def test_extreme_values_are_exact(lnbnn):
    """Rows of 0s and 255s in appearance and location at the largest weight:
    the largest distance, 128 * 255^2 + 48 * 2 * 255^2 = 14,565,600, and every
    mix of extremes comes out exact."""
    vals = [0, 1, 127, 128, 129, 254, 255]
    rows = []
    for a in vals:
        for lx in (0, 128, 255):
            for ly in (0, 255):
                r = np.full(130, a, np.uint8)
                r[128], r[129] = lx, ly
                rows.append(r)
    ref = np.array(rows, np.uint8)
    rng = np.random.default_rng(7)
    mixed = rng.choice(np.array([0, 255], np.uint8), size=(64, 130))
    ref = np.concatenate([ref, mixed])
    q = np.concatenate([ref[::3], rng.choice(np.array([0, 255], np.uint8), size=(40, 130))])
    labels = (np.arange(len(ref)) % 3).astype(np.int32)
    with lnbnn.Index(dev(ref), dev(labels), 3, location_weight=48) as ix:
        idx, dist = ix.knn_search(dev(q), len(ref))  # every distance of every query
        ix.sync()
    od, oj = oracle.knn(ref, q, len(ref), location_weight=48)
    assert np.array_equal(dist.cpu().numpy(), od) and np.array_equal(idx.cpu().numpy(), oj)
    assert od.max() == 8323200 + 48 * 2 * 255 ** 2


def test_ties_many_splits_and_logodds(lnbnn):
    # few distinct values: many ties; a small query batch runs with many reference splits
    ref, labels, q = located_case(120, 70000, 90, 5, hi=3, loc_hi=4)
    off = np.array([0, 30, 90], np.int64)
    with lnbnn.Index(dev(ref), dev(labels), 5, location_weight=3) as ix:
        assert ix.plan_splits(len(q)) > 1
        idx, dist = ix.knn_search(dev(q), 12)
        t, c = ix.lnbnn_classify(dev(q), dev(off), 11)
        lt, lc, ln = ix.nbnn_logodds_classify(dev(q), dev(off), 0.2, True)
        ix.sync()
    od, oj = oracle.knn(ref, q, 12, location_weight=3)
    assert np.array_equal(idx.cpu().numpy(), oj) and np.array_equal(dist.cpu().numpy(), od)
    ot, oc = oracle.local_nbnn(ref, labels, 5, q, off, 11, location_weight=3)
    assert np.array_equal(t.cpu().numpy(), ot) and np.array_equal(c.cpu().numpy(), oc)
    wt, wc, wn, near = oracle.logodds.nbnn_logodds(ref, labels, 5, q, off, 0.2, True, location_weight=3)
    assert np.all(np.abs(lt.cpu().numpy() - wt) <= 1e-9 * np.maximum(1, np.abs(wt)) + 1e-6 * (near[:, None] + 1))
    assert np.all(np.abs(ln.cpu().numpy() - wn) <= near)


def test_errors_layout_and_file(lnbnn, tmp_path):
    ref, labels, q = located_case(130, 3000, 200, 4)
    off = np.array([0, 200], np.int64)
    for bad in (-1, 49):
        with pytest.raises(lnbnn.LnbnnError) as e:
            lnbnn.Index(dev(ref), dev(labels), 4, location_weight=bad)
        assert e.value.code == 1
    with lnbnn.Index(dev(ref), dev(labels), 4, location_weight=5) as ix:
        with pytest.raises(lnbnn.LnbnnError) as e:
            ix.prepare_fp8()
        assert e.value.code == 8
        with pytest.raises(ValueError):
            ix.knn_search(dev(q[:, :128]), 3)  # 128-byte rows on a located index
        t, c = ix.lnbnn_classify(dev(q), dev(off), 10)
        th, ch = ix.classify_host(q, off, 10)
        ix.sync()
        assert np.array_equal(th, t.cpu().numpy()) and np.array_equal(ch, c.cpu().numpy())
        path = str(tmp_path / "located.lnbnn")
        ix.save(path)
    with lnbnn.Index.load(path) as ix2:
        assert (ix2.row_bytes, ix2.location_weight) == (130, 5)
        t2, c2 = ix2.lnbnn_classify(dev(q), dev(off), 10)
        ix2.sync()
        assert torch.equal(t2, t) and torch.equal(c2, c)


def test_caltech101_located_full_size_sampled(lnbnn):
    """The 101-class index (1.515M references) with locations, weight 10 (alpha
    about 3 grid cells), all 200 query images in one call; sampled rows and one
    whole image against the oracle."""
    from paper_1112_0059_gb300 import synth
    w = synth.workload("caltech101-like")
    ref, labels = synth.reference_set(w)
    q, off, _ = synth.query_set(w)
    ref = synth.located(ref, synth.reference_locations(w))
    q = synth.located(q, synth.query_locations(w))
    rng = np.random.default_rng(23)
    rows = np.unique(np.concatenate([[0, len(q) - 1], rng.integers(0, len(q), size=14)]))
    with lnbnn.Index(dev(ref), dev(labels), w.n_classes, location_weight=10) as ix:
        qd = dev(q)
        idx, dist = ix.knn_search(qd, 11)
        t, c = ix.lnbnn_classify(qd, dev(off), 10)
        ix.sync()
    od, oj = oracle.knn(ref, q[rows], 11, location_weight=10)
    assert np.array_equal(idx.cpu().numpy()[rows], oj.astype(np.int32))
    assert np.array_equal(dist.cpu().numpy()[rows], od.astype(np.int32))
    img = 77
    qi = q[off[img]:off[img + 1]]
    ot, oc = oracle.local_nbnn(ref, labels, w.n_classes, qi, np.array([0, len(qi)]), 10, location_weight=10)
    assert np.array_equal(t.cpu().numpy()[img], ot[0]) and c.cpu().numpy()[img] == oc[0]
