"""An index saved to a file and loaded back gives the same results."""
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


def test_save_load_round_trip(lnbnn, tmp_path):
    rng = np.random.default_rng(95)
    ref = rng.integers(0, 256, size=(9000, 128), dtype=np.uint8)
    labels = rng.permutation(np.arange(9000) % 7).astype(np.int32)  # not grouped: a class-sorted copy too
    q = rng.integers(0, 256, size=(400, 128), dtype=np.uint8)
    off = np.array([0, 150, 400], np.int64)
    qd, od = torch.from_numpy(q).cuda(), torch.from_numpy(off).cuda()
    path = str(tmp_path / "index.lnbnn")
    with lnbnn.Index(torch.from_numpy(ref).cuda(), torch.from_numpy(labels).cuda(), 7) as ix:
        want = [ix.lnbnn_classify(qd, od, 10), ix.nbnn_classify(qd, od), ix.knn_search(qd, 11)]
        ix.sync()
        ix.save(path)
    assert (tmp_path / "index.lnbnn").stat().st_size == 32 + 9000 * 128 + 9000 * 4 + 8
    with lnbnn.Index.load(path) as ix:
        assert ix.n_ref == 9000 and ix.n_classes == 7
        got = [ix.lnbnn_classify(qd, od, 10), ix.nbnn_classify(qd, od), ix.knn_search(qd, 11)]
        ix.prepare_fp8()
        ft, fc = ix.lnbnn_classify(qd, od, 10, shortlist=32)
        ix.sync()
    for (a0, a1), (b0, b1) in zip(want, got):
        assert torch.equal(a0, b0) and torch.equal(a1, b1)
    ot, oc = oracle.local_nbnn(ref, labels, 7, q, off, 10)
    assert np.array_equal(got[0][0].cpu().numpy(), ot) and np.array_equal(got[0][1].cpu().numpy(), oc)
    ct, cc = oracle.local_nbnn_coarse(ref, labels, 7, q, off, 10, 32)
    assert np.array_equal(ft.cpu().numpy(), ct) and np.array_equal(fc.cpu().numpy(), cc)
