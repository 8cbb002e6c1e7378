"""Full-size parity on the 256-class workload: 11.52M reference descriptors,
500 query images x 1,500 descriptors, the launch configuration the benchmark
times (every query row in one call; one reference split for the exact scan at
k = 10).

Each search runs over all 750,000 query rows on the GPU, so the list kind and
schedule are the full-size ones (asserted through lnbnn_plan_search); the
oracle then checks sampled rows (kNN) or whole images (class totals), bit for
bit.  An identity of Algorithm 2's update (Local NBNN totals = sum over
descriptors of min(0, NN_C - dist_B): a class absent from the k nearest has
NN_C >= dist_B) ties the NBNN scan, the kNN scan and the Local NBNN update
together over 50 whole images.
"""
import numpy as np
import pytest

import oracle
from paper_1112_0059_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _sample_rows(M, n, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, M - 1], rng.integers(0, M, size=n)]))


@pytest.fixture(scope="module")
def full():
    from paper_1112_0059_gb300 import build, lnbnn
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    lnbnn.load_library()
    w = synth.workload("caltech256-like")
    ref, labels = synth.reference_set(w)
    q, off, _ = synth.query_set(w)
    ix = lnbnn.Index(dev(ref), dev(labels), w.n_classes)
    qd, offd = dev(q), dev(off)
    yield {"w": w, "ref": ref, "labels": labels, "q": q, "off": off, "ix": ix, "qd": qd, "offd": offd}
    ix.close()


def _knn_full_size(full, k1, rows):
    ix, q = full["ix"], full["q"]
    idx, dist = ix.knn_search(full["qd"], k1)
    ix.sync()
    od, oj = oracle.knn(full["ref"], q[rows], k1)
    assert np.array_equal(dist.cpu().numpy()[rows], od.astype(np.int32))
    assert np.array_equal(idx.cpu().numpy()[rows], oj.astype(np.int32))


def test_k10_register_lists_sampled(full):
    plan = full["ix"].plan_search(len(full["q"]), 11)
    assert plan["splits"] == 1 and plan["list_storage"] == "registers" and plan["list_capacity"] == 16
    _knn_full_size(full, 11, _sample_rows(len(full["q"]), 30, 11))


def test_k50_register_lists_of_64_sampled(full):
    # one split of 11.52M references: the 64-entry lists live in registers
    plan = full["ix"].plan_search(len(full["q"]), 51)
    assert plan["splits"] == 1 and plan["split_len"] > (8 << 20)
    assert plan["list_storage"] == "registers" and plan["list_capacity"] == 64
    _knn_full_size(full, 51, _sample_rows(len(full["q"]), 30, 51))


def test_k100_heap_sampled(full):
    # heaps: eight splits run one after another, each starting from the
    # previous split's heaps of its rows
    plan = full["ix"].plan_search(len(full["q"]), 101)
    assert plan["splits"] == 8 and plan["bound_per_tile"] == 0 and plan["list_storage"] == "global-memory heap"
    _knn_full_size(full, 101, _sample_rows(len(full["q"]), 30, 101))


def test_whole_images_local_and_nbnn(full):
    """Alg. 2 and Alg. 1 on the whole batch; two whole images through the oracle."""
    ix, q, off, w = full["ix"], full["q"], full["off"], full["w"]
    lt, lc = ix.lnbnn_classify(full["qd"], full["offd"], 10)
    nt, nc = ix.nbnn_classify(full["qd"], full["offd"])
    ix.sync()
    lt, lc, nt, nc = lt.cpu().numpy(), lc.cpu().numpy(), nt.cpu().numpy(), nc.cpu().numpy()
    for img in (0, 317):
        qi = q[off[img]:off[img + 1]]
        one = np.array([0, len(qi)])
        ot, oc = oracle.local_nbnn(full["ref"], full["labels"], w.n_classes, qi, one, 10)
        assert np.array_equal(lt[img], ot[0]) and lc[img] == oc[0]
        ont, onc = oracle.nbnn(full["ref"], full["labels"], w.n_classes, qi, one)
        assert np.array_equal(nt[img], ont[0]) and nc[img] == onc[0]
    assert (lt <= 0).all() and (nt >= 0).all()


def test_local_update_identity_over_50_images(full):
    """Local totals == sum_i min(0, NN_C(i) - dist_B(i)) with NN_C from the NBNN
    scan (one descriptor per image) and dist_B the (k+1)-th distance of the kNN
    scan: three kernels' outputs tied together exactly, at full size."""
    ix, off, k = full["ix"], full["off"], 10
    n_img = 50
    m = int(off[n_img])
    qd = full["qd"][:m]
    per_row = torch.arange(m + 1, dtype=torch.int64, device="cuda")
    nn_c, _ = ix.nbnn_classify(qd, per_row)                     # [m, C]: NN_C of each descriptor
    _, dist = ix.knn_search(qd, k + 1)                          # [m, k+1]
    lt, lc = ix.lnbnn_classify(qd, full["offd"][:n_img + 1], k)  # [50, C]
    ix.sync()
    nn_c = nn_c.cpu().numpy()
    dist_b = dist.cpu().numpy()[:, k].astype(np.int64)
    inc = np.minimum(0, nn_c - dist_b[:, None])
    want = np.add.reduceat(inc, off[:n_img], axis=0)
    assert np.array_equal(lt.cpu().numpy(), want)
    cls = np.argmin(want, axis=1)  # lowest class on ties, as the paper's argmin is read here
    assert np.array_equal(lc.cpu().numpy(), cls)


def test_fp8_shortlist_sampled_and_one_image(full):
    """The FP8 shortlist form in the bench's launch configuration against the
    oracle's coarse form (bit-exact) and its recall against the exact oracle."""
    ix, q, off, w = full["ix"], full["q"], full["off"], full["w"]
    ix.prepare_fp8()
    m = 24  # the benchmark's shortlist
    plan = ix.plan_search(len(q), m, fp8=True)
    assert plan["splits"] >= 1 and plan["list_capacity"] == 24
    rows = _sample_rows(len(q), 30, 21)
    idx, dist = ix.knn_search(full["qd"], 11, shortlist=m)
    t, c = ix.lnbnn_classify(full["qd"], full["offd"], 10, shortlist=m)
    ix.sync()
    od, oj = oracle.knn_coarse(full["ref"], q[rows], 11, m)
    assert np.array_equal(idx.cpu().numpy()[rows], oj.astype(np.int32))
    assert np.array_equal(dist.cpu().numpy()[rows], od.astype(np.int32))
    ed, ej = oracle.knn(full["ref"], q[rows], 11)
    recall = np.mean([len(set(a) & set(b)) / 11 for a, b in zip(oj, ej)])
    assert recall >= 0.99
    img = 123
    qi = q[off[img]:off[img + 1]]
    ot, oc = oracle.local_nbnn_coarse(full["ref"], full["labels"], w.n_classes, qi, np.array([0, len(qi)]), 10, m)
    assert np.array_equal(t.cpu().numpy()[img], ot[0]) and c.cpu().numpy()[img] == oc[0]
