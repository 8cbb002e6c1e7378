"""FP8 E4M3 shortlist search on the GPU against the oracle's coarse-shortlist
form: bit-exact neighbours, distances and Local NBNN totals; the reduction to
the exact search when the shortlist holds every reference; recall on
SIFT-like data; independence of the batch a query is searched in."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def uniform_case(seed, N, M, C, lo=0, hi=256):
    rng = np.random.default_rng(seed)
    ref = rng.integers(lo, hi, size=(N, 128)).astype(np.uint8)
    q = rng.integers(lo, hi, size=(M, 128)).astype(np.uint8)
    labels = rng.integers(0, C, size=N).astype(np.int32)
    labels[:C] = np.arange(C)
    return ref, labels, q


def sift_case(classes=12, ref_imgs=4, ref_desc=400, q_imgs=6):
    from paper_1112_0059_gb300 import synth
    w = dataclasses.replace(synth.workload("caltech256-like"), n_classes=classes, ref_imgs_per_class=ref_imgs,
                            ref_desc_per_img=ref_desc, n_query_imgs=q_imgs, query_counts=("fixed", 150))
    ref, labels = synth.reference_set(w)
    q, off, _ = synth.query_set(w)
    return ref, labels, q, off, classes


@pytest.mark.parametrize("shortlist", [16, 24, 32, 64])
@pytest.mark.parametrize("data", ["uniform", "sift"])
def test_knn_fp8_matches_oracle(lnbnn, shortlist, data):
    # ragged: N not a multiple of the 256-row tile, M not a multiple of 128
    if data == "uniform":
        ref, labels, q = uniform_case(40 + shortlist, 5037, 301, 5)
    else:
        ref, labels, q, _, _ = sift_case()
        q = q[:301]
    with lnbnn.Index(dev(ref), dev(labels), int(labels.max()) + 1) as ix:
        ix.prepare_fp8()
        for k in (1, 10):
            idx, dist = ix.knn_search(dev(q), k, shortlist=shortlist)
            ix.sync()
            od, oj = oracle.knn_coarse(ref, q, k, shortlist)
            assert np.array_equal(idx.cpu().numpy(), oj), f"k={k}"
            assert np.array_equal(dist.cpu().numpy(), od), f"k={k}"


@pytest.mark.parametrize("shortlist", [11, 32, 100])
def test_lnbnn_fp8_matches_oracle(lnbnn, shortlist):
    ref, labels, q, off, C = sift_case()
    with lnbnn.Index(dev(ref), dev(labels), C) as ix:
        ix.prepare_fp8()
        t, c = ix.lnbnn_classify(dev(q), dev(off), 10, shortlist=shortlist)
        ix.sync()
        ot, oc = oracle.local_nbnn_coarse(ref, labels, C, q, off, 10, shortlist)
        assert np.array_equal(t.cpu().numpy(), ot) and np.array_equal(c.cpu().numpy(), oc)


def test_full_shortlist_is_the_exact_search(lnbnn):
    ref, labels, q = uniform_case(50, 240, 200, 4, hi=8)  # few values: many ties
    off = np.array([0, 37, 37, 200], np.int64)
    with lnbnn.Index(dev(ref), dev(labels), 4) as ix:
        ix.prepare_fp8()
        idx, dist = ix.knn_search(dev(q), 12, shortlist=256)  # > N: every reference
        t, c = ix.lnbnn_classify(dev(q), dev(off), 5, shortlist=240)
        ix.sync()
        od, oj = oracle.knn(ref, q, 12)
        assert np.array_equal(idx.cpu().numpy(), oj) and np.array_equal(dist.cpu().numpy(), od)
        ot, oc = oracle.local_nbnn(ref, labels, 4, q, off, 5)
        assert np.array_equal(t.cpu().numpy(), ot) and np.array_equal(c.cpu().numpy(), oc)


def test_recall_on_sift_like_data(lnbnn):
    ref, labels, q, off, C = sift_case(classes=16, ref_imgs=6, ref_desc=500, q_imgs=8)
    with lnbnn.Index(dev(ref), dev(labels), C) as ix:
        ix.prepare_fp8()
        idx, _ = ix.knn_search(dev(q), 11, shortlist=32)
        t, c = ix.lnbnn_classify(dev(q), dev(off), 10, shortlist=32)
        ix.sync()
    _, oj = oracle.knn(ref, q, 11)
    got = idx.cpu().numpy()
    recall = np.mean([len(set(got[i]) & set(oj[i])) / 11 for i in range(len(q))])
    assert recall >= 0.999, recall
    ot, oc = oracle.local_nbnn(ref, labels, C, q, off, 10)
    assert np.array_equal(c.cpu().numpy(), oc)
    rel = np.abs(t.cpu().numpy() - ot).sum() / np.abs(ot).sum()
    assert rel < 1e-3, rel


def test_result_does_not_depend_on_the_batch(lnbnn):
    # a small call runs with many reference splits, a large one with few;
    # a query's shortlist (and so its result) must be the same
    ref, labels, q = uniform_case(60, 70000, 2000, 6)
    with lnbnn.Index(dev(ref), dev(labels), 6) as ix:
        ix.prepare_fp8()
        big_i, big_d = ix.knn_search(dev(q), 10, shortlist=32)
        small_i, small_d = ix.knn_search(dev(q[:100]), 10, shortlist=32)
        ix.sync()
        assert np.array_equal(big_i.cpu().numpy()[:100], small_i.cpu().numpy())
        assert np.array_equal(big_d.cpu().numpy()[:100], small_d.cpu().numpy())
        od, oj = oracle.knn_coarse(ref, q[:100], 10, 32)
        assert np.array_equal(small_i.cpu().numpy(), oj) and np.array_equal(small_d.cpu().numpy(), od)


def test_errors_and_workspace(lnbnn):
    ref, labels, q = uniform_case(70, 3000, 260, 3)
    off = np.array([0, 100, 260], np.int64)
    with lnbnn.Index(dev(ref), dev(labels), 3) as ix:
        with pytest.raises(lnbnn.LnbnnError) as e:
            ix.knn_search(dev(q), 5, shortlist=16)
        assert e.value.code == 11  # no FP8 operand yet
        ix.prepare_fp8()
        ix.prepare_fp8()  # repeated: no-op
        with pytest.raises(lnbnn.LnbnnError) as e:
            ix.lnbnn_classify(dev(q), dev(off), 10, shortlist=10)  # needs k + 1 <= shortlist
        assert e.value.code == 4
        with pytest.raises(lnbnn.LnbnnError) as e:
            ix.knn_search(dev(q), 5, shortlist=257)
        assert e.value.code == 4
        with ix.workspace(300, 15) as ws:  # holds shortlists up to 16
            t, c = ix.lnbnn_classify(dev(q), dev(off), 10, shortlist=16, workspace=ws)
            ix.sync()
            ot, oc = oracle.local_nbnn_coarse(ref, labels, 3, q, off, 10, 16)
            assert np.array_equal(t.cpu().numpy(), ot) and np.array_equal(c.cpu().numpy(), oc)
            with pytest.raises(lnbnn.LnbnnError) as e:
                ix.lnbnn_classify(dev(q), dev(off), 10, shortlist=32, workspace=ws)
            assert e.value.code == 10
        # host-buffer form
        th, ch = ix.classify_host(q, off, 10, shortlist=16)
        assert np.array_equal(th, ot) and np.array_equal(ch, oc)


# ------------------------------------------------------------------ full-size workloads (sampled)

def _sample_rows(M, n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, M - 1], rng.integers(0, M, size=n)]))


def test_fp8_caltech101_full_size(lnbnn):
    from paper_1112_0059_gb300 import synth
    w = synth.workload("caltech101-like")
    ref, labels = synth.reference_set(w)
    q, off, _ = synth.query_set(w)
    rows = _sample_rows(len(q), 16, 22)
    with lnbnn.Index(dev(ref), dev(labels), w.n_classes) as ix:
        ix.prepare_fp8()
        qd = dev(q)
        for m in (16, 64):
            idx, dist = ix.knn_search(qd, 11, shortlist=m)
            ix.sync()
            od, oj = oracle.knn_coarse(ref, q[rows], 11, m)
            assert np.array_equal(idx.cpu().numpy()[rows], oj.astype(np.int32)), m
            assert np.array_equal(dist.cpu().numpy()[rows], od.astype(np.int32)), m
        t, c = ix.lnbnn_classify(qd, dev(off), 10, shortlist=32)
        ix.sync()
    img = 37  # one whole image through the oracle
    qi = q[off[img]:off[img + 1]]
    ot, oc = oracle.local_nbnn_coarse(ref, labels, w.n_classes, qi, np.array([0, len(qi)]), 10, 32)
    assert np.array_equal(t.cpu().numpy()[img], ot[0]) and c.cpu().numpy()[img] == oc[0]
    assert (t.cpu().numpy() <= 0).all()
