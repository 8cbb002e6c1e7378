"""NBNN as a sum of log-odds increments (Section 3.1) on the GPU against the
float64 oracle: per-image totals within float64 rounding, the same number of
positive increments and the same class wherever the decision is clear of
rounding; the degenerate cases; independence of the batch."""
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


def assert_matches(got, want, beta, dmax):
    """got/want = (totals, classes, counts[, near]).  Totals agree to float64
    rounding (each increment is a difference of terms up to beta * dmax);
    counts differ at most by the increments within the oracle's decision
    tolerance of 0; classes agree where the top two totals are further apart
    than the totals' tolerance."""
    t, c, n = (x.cpu().numpy() for x in got[:3])
    ot, oc, on, near = want
    tol_inc = 1e-9 * (1.0 + beta * dmax)
    scale = np.maximum(1.0, np.abs(ot))
    assert np.all(np.abs(t - ot) <= 1e-11 * scale + tol_inc * (near[:, None] + 1)), np.abs(t - ot).max()
    assert np.all(np.abs(n - on) <= near), (n, on, near)
    for g in range(len(oc)):
        srt = np.sort(ot[g])[::-1]
        if len(srt) < 2 or srt[0] - srt[1] > 1e-9 * max(1.0, abs(srt[0])) + tol_inc * (near[g] + 1):
            assert c[g] == oc[g], (g, c[g], oc[g])


def uniform_case(seed, N, sizes, C):
    rng = np.random.default_rng(seed)
    ref = rng.integers(0, 256, size=(N, 128)).astype(np.uint8)
    labels = rng.integers(0, C, size=N).astype(np.int32)
    labels[:C] = np.arange(C)
    q = rng.integers(0, 256, size=(int(sum(sizes)), 128)).astype(np.uint8)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return ref, labels, q, off


@pytest.mark.parametrize("positive_only", [False, True])
@pytest.mark.parametrize("beta", [0.0, 1e-5, 3e-4, 1.0])
def test_matches_oracle(lnbnn, beta, positive_only):
    # ragged: N not a multiple of 256, M = 301 not a multiple of 128, an empty image
    ref, labels, q, off = uniform_case(90, 5037, [120, 0, 1, 180], 5)
    with lnbnn.Index(dev(ref), dev(labels), 5) as ix:
        got = ix.nbnn_logodds_classify(dev(q), dev(off), beta, positive_only)
        ix.sync()
    want = oracle.logodds.nbnn_logodds(ref, labels, 5, q, off, beta, positive_only)
    dmax = float(oracle.class_min(ref, labels, 5, q).max())
    assert_matches(got, want, beta, dmax)
    t, c, n = (x.cpu().numpy() for x in got)
    assert (t[1] == 0).all() and c[1] == 0 and n[1] == 0  # the empty image
    if beta == 0.0:
        assert (t == 0).all() and (c == 0).all()
        assert np.array_equal(n, np.zeros(4) if positive_only else np.diff(off) * 5)
    if not positive_only:
        assert np.array_equal(n, np.diff(off) * 5)


def sift_case(classes=12, ref_imgs=4, ref_desc=400, q_imgs=6, per_img=150):
    from paper_1112_0059_gb300 import synth
    w = dataclasses.replace(synth.workload("caltech256-like"), n_classes=classes, ref_imgs_per_class=ref_imgs,
                            ref_desc_per_img=ref_desc, n_query_imgs=q_imgs, query_counts=("fixed", per_img))
    ref, labels = synth.reference_set(w)
    q, off, _ = synth.query_set(w)
    return ref, labels, q, off, classes


def test_sift_like_positive_increments(lnbnn):
    """On SIFT-like data, a beta at which about half of the increments are
    positive (the regime of Table 1): same totals, counts and classes."""
    ref, labels, q, off, C = sift_case()
    D = oracle.class_min(ref, labels, C, q)
    beta = 1.0 / float(np.median(D.max(axis=1) - D.min(axis=1)))
    with lnbnn.Index(dev(ref), dev(labels), C) as ix:
        for positive_only in (True, False):
            got = ix.nbnn_logodds_classify(dev(q), dev(off), beta, positive_only)
            ix.sync()
            want = oracle.logodds.nbnn_logodds(ref, labels, C, q, off, beta, positive_only)
            assert_matches(got, want, beta, float(D.max()))
            if positive_only:
                frac = got[2].cpu().numpy().sum() / (len(q) * C)
                assert 0.05 < frac < 0.95, frac


def test_ties_and_batch_independence(lnbnn):
    # few distinct values: many classes tie at the nearest distance
    rng = np.random.default_rng(91)
    ref = rng.integers(0, 3, size=(600, 128)).astype(np.uint8)
    labels = (np.arange(600) % 7).astype(np.int32)
    q = rng.integers(0, 3, size=(260, 128)).astype(np.uint8)
    off = np.array([0, 40, 41, 200, 260], np.int64)
    with lnbnn.Index(dev(ref), dev(labels), 7) as ix:
        for beta, pos in ((0.05, True), (0.05, False), (2.0, True)):
            t, c, n = ix.nbnn_logodds_classify(dev(q), dev(off), beta, pos)
            ix.sync()
            want = oracle.logodds.nbnn_logodds(ref, labels, 7, q, off, beta, pos)
            assert_matches((t, c, n), want, beta, float(oracle.class_min(ref, labels, 7, q).max()))
            for g in range(len(off) - 1):
                qi = dev(q[off[g]:off[g + 1]])
                t1, c1, n1 = ix.nbnn_logodds_classify(qi, dev(np.array([0, off[g + 1] - off[g]])), beta, pos)
                ix.sync()
                assert torch.equal(t1[0], t[g]) and torch.equal(c1[0], c[g]) and torch.equal(n1[0], n[g]), g


def test_errors_and_workspace(lnbnn):
    ref, labels, q, off = uniform_case(92, 900, [100, 160], 3)
    with lnbnn.Index(dev(ref), dev(labels), 3) as ix:
        for bad in (-1.0, float("nan"), float("inf"), 1e300):
            with pytest.raises(lnbnn.LnbnnError) as e:
                ix.nbnn_logodds_classify(dev(q), dev(off), bad)
            assert e.value.code == 1, bad
        t, c, n = ix.nbnn_logodds_classify(dev(q), dev(off), 1e-4, True)
        with ix.workspace(300, 10) as ws:
            t2, c2, n2 = ix.nbnn_logodds_classify(dev(q), dev(off), 1e-4, True, workspace=ws)
            ix.sync()
            assert torch.equal(t, t2) and torch.equal(c, c2) and torch.equal(n, n2)
    with lnbnn.Index(dev(ref), dev(np.zeros(900, np.int32)), 1) as ix:  # one class: no complement
        with pytest.raises(lnbnn.LnbnnError) as e:
            ix.nbnn_logodds_classify(dev(q), dev(off), 1e-4)
        assert e.value.code == 1


def test_caltech101_full_size_one_image(lnbnn):
    """The 101-class index (1.515M references) with all 200 query images in one
    call; one whole image against the oracle, the rest against properties."""
    from paper_1112_0059_gb300 import synth
    w = synth.workload("caltech101-like")
    ref, labels = synth.reference_set(w)
    q, off, _ = synth.query_set(w)
    img = 123
    qi = q[off[img]:off[img + 1]]
    Di = oracle.class_min(ref, labels, w.n_classes, qi)
    beta = 1.0 / float(np.median(Di.max(axis=1) - Di.min(axis=1)))
    with lnbnn.Index(dev(ref), dev(labels), w.n_classes) as ix:
        t, c, n = ix.nbnn_logodds_classify(dev(q), dev(off), beta, True)
        s_nbnn, _ = ix.nbnn_classify(dev(q), dev(off))
        ix.sync()
    ot, oc, on, near = oracle.logodds.nbnn_logodds(ref, labels, w.n_classes, qi, np.array([0, len(qi)]), beta, True)
    assert_matches((t[img:img + 1], c[img:img + 1], n[img:img + 1]), (ot, oc, on, near), beta, float(Di.max()))
    n = n.cpu().numpy()
    assert (n > 0).all() and (n < np.diff(off) * w.n_classes).all()
    assert (t.cpu().numpy() >= 0).all()  # only positive increments were added
