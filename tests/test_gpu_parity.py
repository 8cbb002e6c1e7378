"""CUDA path against the CPU oracle, element by element, through the C ABI.

Bar (exact integer work): neighbour rows, int32 distances, int64 totals and
chosen classes are bit-identical to the oracle.  Small cases span several
query tiles (128 rows) and reference tiles (256 rows) with ragged tails; the
full-size workloads are compared on sampled rows (and one whole image) in the
launch configuration the benchmark times.
"""
import numpy as np
import pytest

import oracle
from paper_1112_0059_gb300 import synth

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


def make_index(lnbnn, ref, labels, C):
    return lnbnn.Index(dev(ref), dev(labels.astype(np.int32)), C)


def check_knn(ix, ref, q, k):
    idx, dist = ix.knn_search(dev(q), k)
    torch.cuda.synchronize()
    ix.sync()
    od, oj = oracle.knn(ref, q, k)
    assert np.array_equal(dist.cpu().numpy(), od.astype(np.int32))
    assert np.array_equal(idx.cpu().numpy(), oj.astype(np.int32))


def check_classify(ix, ref, labels, C, q, offsets, k):
    lt, lc = ix.lnbnn_classify(dev(q), dev(offsets), k)
    nt, nc = ix.nbnn_classify(dev(q), dev(offsets))
    ix.sync()
    ot, oc = oracle.local_nbnn(ref, labels, C, q, offsets, k)
    assert np.array_equal(lt.cpu().numpy(), ot)
    assert np.array_equal(lc.cpu().numpy(), oc)
    ont, onc = oracle.nbnn(ref, labels, C, q, offsets)
    assert np.array_equal(nt.cpu().numpy(), ont)
    assert np.array_equal(nc.cpu().numpy(), onc)


def random_case(seed, N, M, C, hi=256, dims=128, n_img=3):
    rng = np.random.default_rng(seed)
    ref = np.zeros((N, 128), np.uint8)
    q = np.zeros((M, 128), np.uint8)
    cols = rng.choice(128, size=dims, replace=False)
    ref[:, cols] = rng.integers(0, hi, size=(N, dims))
    q[:, cols] = rng.integers(0, hi, size=(M, dims))
    labels = rng.integers(0, C, size=N).astype(np.int32)
    labels[:C] = np.arange(C)
    cuts = np.sort(rng.integers(0, M + 1, size=n_img - 1))
    offsets = np.concatenate([[0], cuts, [M]]).astype(np.int64)
    return ref, labels, q, offsets


# ------------------------------------------------------------------ tiny workload

def test_tiny_workload_bit_exact(lnbnn):
    w = synth.workload("tiny")
    ref, labels = synth.reference_set(w)
    q, off, _ = synth.query_set(w)
    with make_index(lnbnn, ref, labels, w.n_classes) as ix:
        check_knn(ix, ref, q, 11)
        check_classify(ix, ref, labels, w.n_classes, q, off, 10)


@pytest.mark.parametrize("k", [1, 2, 10, 50, 100, 255])
def test_k_range(lnbnn, k):
    ref, labels, q, off = random_case(1, 3000 + 37, 300 + 5, 7)
    with make_index(lnbnn, ref, labels, 7) as ix:
        check_knn(ix, ref, q, k)
        if k + 1 <= len(ref):
            check_classify(ix, ref, labels, 7, q, off, k)


@pytest.mark.parametrize("K1", [15, 16, 17, 24, 25, 32, 33, 64, 65])
def test_list_kind_boundaries_many_splits(lnbnn, K1):
    # k+1 at the edges of the list kinds (16- / 24- / 32-entry register lists,
    # 64-entry shared-memory lists, heaps), a small batch over many reference
    # splits (so the lists of a row share a bound) and coordinates with ties;
    # exact search and FP8 shortlists of exactly K1 and of 2 K1
    ref, labels, q, off = random_case(6 + K1, 50000, 150, 5, hi=4, dims=6)
    with make_index(lnbnn, ref, labels, 5) as ix:
        assert ix.plan_splits(len(q)) > 8
        check_knn(ix, ref, q, K1)
        check_classify(ix, ref, labels, 5, q, off, K1 - 1)
        ix.prepare_fp8()
        for m in (K1, 2 * K1):
            idx, dist = ix.knn_search(dev(q), K1, shortlist=m)
            ix.sync()
            od, oj = oracle.knn_coarse(ref, q, K1, m)
            assert np.array_equal(idx.cpu().numpy(), oj) and np.array_equal(dist.cpu().numpy(), od), m


@pytest.mark.parametrize("N,M", [(1, 1), (2, 3), (255, 129), (256, 128), (257, 127), (1000, 1), (4099, 1030)])
def test_ragged_shapes(lnbnn, N, M):
    ref, labels, q, off = random_case(2, N, M, 1 if N < 3 else 3, n_img=2)
    with make_index(lnbnn, ref, labels, 1 if N < 3 else 3) as ix:
        check_knn(ix, ref, q, min(N, 5))
        if N >= 2:
            check_classify(ix, ref, labels, 1 if N < 3 else 3, q, off, min(N - 1, 4))


def test_many_splits_small_batch(lnbnn):
    # one query tile against 60k references: the search splits the reference set
    ref, labels, q, off = random_case(3, 60000, 64, 5)
    with make_index(lnbnn, ref, labels, 5) as ix:
        check_knn(ix, ref, q, 20)
        check_classify(ix, ref, labels, 5, q, off, 10)


def test_shared_row_bound_with_ties(lnbnn):
    # one query tile against 90k references: many splits, so the lists of a row
    # share a bound and leave out columns beyond it; coordinates in {0..2} on
    # a few dims put many columns exactly at the bound, where the lower row
    # must still win (exact and FP8 shortlist, 16- and 32-entry lists)
    for hi, dims in ((3, 5), (256, 128)):
        ref, labels, q, off = random_case(5, 90000, 100, 6, hi=hi, dims=dims)
        with make_index(lnbnn, ref, labels, 6) as ix:
            assert ix.plan_splits(len(q)) > 8
            for k in (1, 15, 31):
                check_knn(ix, ref, q, k)
            check_classify(ix, ref, labels, 6, q, off, 10)
            ix.prepare_fp8()
            for m in (16, 32):
                idx, dist = ix.knn_search(dev(q), 11, shortlist=m)
                ix.sync()
                od, oj = oracle.knn_coarse(ref, q, 11, m)
                assert np.array_equal(idx.cpu().numpy(), oj) and np.array_equal(dist.cpu().numpy(), od), (hi, m)


def test_randomized_shapes_against_oracle(lnbnn):
    # random sizes (one query tile or a few, up to many reference splits), value
    # ranges from heavy ties to full range, k across the 16- and 32-entry lists;
    # every result bit-exact with the oracle, and the same when searched again
    rng = np.random.default_rng(77)
    for case in range(16):
        N = int(rng.integers(300, 40000))
        M = int(rng.integers(1, 400))
        hi = int(rng.choice([2, 3, 8, 256]))
        dims = int(rng.choice([3, 16, 128]))
        C = int(rng.integers(1, 9))
        k = int(rng.integers(1, min(31, N - 1) + 1))
        ref, labels, q, off = random_case(1000 + case, N, M, C, hi=hi, dims=dims)
        with make_index(lnbnn, ref, labels, C) as ix:
            check_knn(ix, ref, q, k)
            a = ix.knn_search(dev(q), k)
            b = ix.knn_search(dev(q), k)
            ix.sync()
            assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), case
            if k + 1 <= N:
                check_classify(ix, ref, labels, C, q, off, k)


# ------------------------------------------------------------------ adversarial ties

def test_ties_small_values(lnbnn):
    # coordinates in {0..3} on 4 dims: massive distance ties, lowest row must win
    ref, labels, q, off = random_case(4, 2000, 300, 4, hi=4, dims=4)
    with make_index(lnbnn, ref, labels, 4) as ix:
        check_knn(ix, ref, q, 30)
        check_classify(ix, ref, labels, 4, q, off, 10)


def test_duplicates_zeros_and_self_queries(lnbnn):
    rng = np.random.default_rng(5)
    ref = rng.integers(0, 256, size=(700, 128)).astype(np.uint8)
    ref[100:140] = 0
    ref[300:310] = ref[5]
    labels = (np.arange(700) % 6).astype(np.int32)
    q = np.concatenate([ref[[5, 120, 300, 699]], np.zeros((3, 128), np.uint8),
                        rng.integers(0, 256, size=(20, 128)).astype(np.uint8)])
    off = np.array([0, 4, 7, 27], np.int64)
    with make_index(lnbnn, ref, labels, 6) as ix:
        check_knn(ix, ref, q, 45)
        check_classify(ix, ref, labels, 6, q, off, 12)


def test_extreme_values_exact(lnbnn):
    # all-255 against all-0 gives the largest distance 128 * 255^2 = 8,323,200
    ref = np.zeros((600, 128), np.uint8)
    ref[::2] = 255
    ref[1::3, :64] = 255
    labels = (np.arange(600) % 3).astype(np.int32)
    q = np.stack([np.full(128, 255, np.uint8), np.zeros(128, np.uint8),
                  np.r_[np.full(64, 255), np.zeros(64)].astype(np.uint8)])
    with make_index(lnbnn, ref, labels, 3) as ix:
        check_knn(ix, ref, q, 255)
        check_classify(ix, ref, labels, 3, q, np.array([0, 1, 3], np.int64), 20)


def test_unsorted_labels(lnbnn):
    # labels interleaved: NBNN uses a class-sorted copy, kNN rows keep the caller's order
    ref, labels, q, off = random_case(6, 5000, 500, 9)
    perm = np.random.default_rng(6).permutation(len(ref))
    ref, labels = ref[perm], labels[perm]
    with make_index(lnbnn, ref, labels, 9) as ix:
        check_knn(ix, ref, q, 11)
        check_classify(ix, ref, labels, 9, q, off, 10)


# ------------------------------------------------------------------ API behaviour

def test_empty_images_and_host_api(lnbnn):
    ref, labels, q, _ = random_case(7, 1500, 200, 4)
    off = np.array([0, 0, 50, 50, 200, 200], np.int64)
    with make_index(lnbnn, ref, labels, 4) as ix:
        check_classify(ix, ref, labels, 4, q, off, 5)
        ht, hc = ix.classify_host(q, off, 5)
        ot, oc = oracle.local_nbnn(ref, labels, 4, q, off, 5)
        assert np.array_equal(ht, ot) and np.array_equal(hc, oc)
        assert ht[0].tolist() == [0, 0, 0, 0] and hc[0] == 0
        nt, nc = ix.classify_host(q, off, None)
        ont, onc = oracle.nbnn(ref, labels, 4, q, off)
        assert np.array_equal(nt, ont) and np.array_equal(nc, onc)


def test_status_codes(lnbnn):
    ref, labels, q, off = random_case(8, 300, 40, 3)
    with make_index(lnbnn, ref, labels, 3) as ix:
        with pytest.raises(lnbnn.LnbnnError) as e:
            ix.lnbnn_classify(dev(q), dev(off), 300)  # k + 1 > N
        assert e.value.code == 4
        with pytest.raises(lnbnn.LnbnnError) as e:
            ix.knn_search(dev(q), 0)
        assert e.value.code == 4
        bad = off.copy()
        bad[-1] = len(q) + 5
        ix.lnbnn_classify(dev(q), dev(bad), 3)
        with pytest.raises(lnbnn.LnbnnError) as e:
            ix.sync()
        assert e.value.code == 9
        ix.sync()  # the error was collected
    with pytest.raises(lnbnn.LnbnnError) as e:
        make_index(lnbnn, ref, np.where(labels == 2, 7, labels), 3)
    assert e.value.code == 2
    with make_index(lnbnn, ref, np.minimum(labels, 1), 3) as ix:  # class 2 has no reference
        with pytest.raises(lnbnn.LnbnnError) as e:
            ix.nbnn_classify(dev(q), dev(off))
        assert e.value.code == 3
        ix.lnbnn_classify(dev(q), dev(off), 3)  # Local NBNN does not need every class
        ix.sync()


def test_repeated_calls_are_stable(lnbnn):
    ref, labels, q, off = random_case(9, 4000, 700, 5)
    with make_index(lnbnn, ref, labels, 5) as ix:
        a = [ix.lnbnn_classify(dev(q), dev(off), 7)[0].cpu().numpy() for _ in range(3)]
        assert all(np.array_equal(a[0], x) for x in a[1:])


# ------------------------------------------------------------------ full-size workloads (sampled)

def _sample_rows(M, n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, M - 1], rng.integers(0, M, size=n)]))


def test_caltech101_like_full_size(lnbnn):
    w = synth.workload("caltech101-like")
    ref, labels = synth.reference_set(w)
    q, off, _ = synth.query_set(w)
    rows = _sample_rows(len(q), 24, 10)
    with make_index(lnbnn, ref, labels, w.n_classes) as ix:
        qd = dev(q)
        for k in (1, 10, 50):
            idx, dist = ix.knn_search(qd, k + 1)
            ix.sync()
            od, oj = oracle.knn(ref, q[rows], k + 1)
            assert np.array_equal(dist.cpu().numpy()[rows], od.astype(np.int32))
            assert np.array_equal(idx.cpu().numpy()[rows], oj.astype(np.int32))
        lt, lc = ix.lnbnn_classify(qd, dev(off), 10)
        nt, nc = ix.nbnn_classify(qd, dev(off))
        ix.sync()
        # one whole image through the oracle
        img = 37
        qi = q[off[img]:off[img + 1]]
        ot, oc = oracle.local_nbnn(ref, labels, w.n_classes, qi, np.array([0, len(qi)]), 10)
        assert np.array_equal(lt.cpu().numpy()[img], ot[0]) and lc.cpu().numpy()[img] == oc[0]
        ont, onc = oracle.nbnn(ref, labels, w.n_classes, qi, np.array([0, len(qi)]))
        assert np.array_equal(nt.cpu().numpy()[img], ont[0]) and nc.cpu().numpy()[img] == onc[0]
        # properties at full size: totals <= 0; the Local totals never exceed 0 and
        # NBNN totals are sums of nonnegative minima
        assert (lt.cpu().numpy() <= 0).all() and (nt.cpu().numpy() >= 0).all()


def test_repeated_searches_with_heavy_ties(lnbnn):
    # Coordinates in {0..2} on 6 dims: most distances tie, and the lists must
    # follow the exact (distance, row) order on every call.
    ref, labels, q, off = random_case(12, 5000 + 11, 700, 4, hi=3, dims=6)
    with make_index(lnbnn, ref, labels, 4) as ix:
        od, oj = oracle.knn(ref, q, 12)
        for _ in range(4):
            idx, dist = ix.knn_search(dev(q), 12)
            ix.sync()
            assert np.array_equal(dist.cpu().numpy(), od.astype(np.int32))
            assert np.array_equal(idx.cpu().numpy(), oj.astype(np.int32))
        for _ in range(2):
            check_classify(ix, ref, labels, 4, q, off, 9)
