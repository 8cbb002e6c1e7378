"""Split-N schedule: the modelled split count, the device autotuner and the
many-list merge change speed only; every schedule gives the oracle's answer."""
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


def test_many_splits_and_autotune(lnbnn):
    rng = np.random.default_rng(80)
    N = 1_300_000  # enough references for 150+ splits of one query tile
    ref = rng.integers(0, 256, size=(N, 128), dtype=np.uint8)
    labels = (np.arange(N) % 9).astype(np.int32)
    q_small = rng.integers(0, 256, size=(100, 128), dtype=np.uint8)
    q_mid = rng.integers(0, 256, size=(1000, 128), dtype=np.uint8)
    with lnbnn.Index(dev(ref), dev(labels), 9) as ix:
        s_small = ix.plan_splits(len(q_small))
        assert s_small > 32, s_small  # one query tile: CTAs on every SM
        before = [ix.knn_search(dev(q), 11) for q in (q_small, q_mid)]
        ix.sync()
        od, oj = oracle.knn(ref, q_small, 11)
        assert np.array_equal(before[0][0].cpu().numpy(), oj) and np.array_equal(before[0][1].cpu().numpy(), od)
        tuned = ix.autotune()
        assert tuned["runs"] >= 10 and tuned["tile_ms"] > 0, tuned
        for n in (1, 100, 1000, 20000, 200000):
            s = ix.plan_splits(n)
            assert 1 <= s <= 2 * torch.cuda.get_device_properties(0).multi_processor_count
        after = [ix.knn_search(dev(q), 11) for q in (q_small, q_mid)]
        ix.sync()
        for (i0, d0), (i1, d1) in zip(before, after):
            assert torch.equal(i0, i1) and torch.equal(d0, d1)
        # a workspace made before tuning still serves every call after it
        with ix.workspace(1000, 10) as ws:
            i2, d2 = ix.knn_search(dev(q_mid), 11, workspace=ws)
            ix.sync()
            assert torch.equal(i2, after[1][0]) and torch.equal(d2, after[1][1])


def test_autotune_on_a_tiny_index(lnbnn):
    rng = np.random.default_rng(81)
    ref = rng.integers(0, 256, size=(100, 128), dtype=np.uint8)  # fewer rows than a query tile
    with lnbnn.Index(dev(ref), dev(np.zeros(100, np.int32)), 1) as ix:
        t = ix.autotune()
        assert t["runs"] == 0
        q = rng.integers(0, 256, size=(7, 128), dtype=np.uint8)
        i, d = ix.knn_search(dev(q), 5)
        ix.sync()
        od, oj = oracle.knn(ref, q, 5)
        assert np.array_equal(i.cpu().numpy(), oj) and np.array_equal(d.cpu().numpy(), od)
