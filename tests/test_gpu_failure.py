"""Failure paths on the GPU without a GPU fault: injected allocation failures
return OOM and leave the library usable; a search whose start gate nothing
opens gives up after its bounded wait, reports TIMEOUT through lnbnn_sync, and
the next call is correct."""
import time

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
    yield lnbnn
    lnbnn.debug_fail_allocations(0)


def case(seed=90, N=6000, M=300, C=4):
    rng = np.random.default_rng(seed)
    ref = rng.integers(0, 256, size=(N, 128), dtype=np.uint8)
    q = rng.integers(0, 256, size=(M, 128), dtype=np.uint8)
    labels = (np.arange(N) % C).astype(np.int32)
    return ref, labels, q


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_injected_allocation_failures(lnbnn):
    ref, labels, q = case()
    for n in (1, 3, 6):  # the first, a middle and a late allocation of index creation
        lnbnn.debug_fail_allocations(n)
        with pytest.raises(lnbnn.LnbnnError) as e:
            lnbnn.Index(dev(ref), dev(labels), 4)
        assert e.value.code == 5
        lnbnn.debug_fail_allocations(0)
    with lnbnn.Index(dev(ref), dev(labels), 4) as ix:
        lnbnn.debug_fail_allocations(1)
        with pytest.raises(lnbnn.LnbnnError) as e:
            ix.workspace(500, 10)
        assert e.value.code == 5
        lnbnn.debug_fail_allocations(1)
        with pytest.raises(lnbnn.LnbnnError) as e:  # the index's own scratch, on first use
            ix.knn_search(dev(q), 5)
        assert e.value.code == 5
        for n in (1, 2):
            lnbnn.debug_fail_allocations(n)
            with pytest.raises(lnbnn.LnbnnError) as e:
                ix.prepare_fp8()
            assert e.value.code == 5
        lnbnn.debug_fail_allocations(0)
        idx, dist = ix.knn_search(dev(q), 5)
        ix.prepare_fp8()
        fi, fd = ix.knn_search(dev(q), 5, shortlist=16)
        ix.sync()
    od, oj = oracle.knn(ref, q, 5)
    assert np.array_equal(idx.cpu().numpy(), oj) and np.array_equal(dist.cpu().numpy(), od)
    cd, cj = oracle.knn_coarse(ref, q, 5, 16)
    assert np.array_equal(fi.cpu().numpy(), cj) and np.array_equal(fd.cpu().numpy(), cd)


def test_start_gate_that_nothing_opens_times_out(lnbnn):
    ref, labels, q = case(91)
    off = np.array([0, 120, 300], np.int64)
    with lnbnn.Index(dev(ref), dev(labels), 4) as ix:
        ix.prepare_fp8()
        gate = torch.zeros(1, dtype=torch.int32, device="cuda")
        ix.set_start_gate(gate)
        calls = [lambda: ix.knn_search(dev(q), 5),
                 lambda: ix.lnbnn_classify(dev(q), dev(off), 10),
                 lambda: ix.nbnn_classify(dev(q), dev(off)),
                 lambda: ix.lnbnn_classify(dev(q), dev(off), 10, shortlist=32)]
        for call in calls:
            t0 = time.perf_counter()
            call()  # launches; the failure is recorded on the device
            with pytest.raises(lnbnn.LnbnnError) as e:
                ix.sync()
            assert e.value.code == 7  # TIMEOUT
            assert 0.5 < time.perf_counter() - t0 < 60
        gate.fill_(1)  # an open gate: normal results
        idx, dist = ix.knn_search(dev(q), 5)
        ix.sync()
        ix.set_start_gate(None)
        t, c = ix.lnbnn_classify(dev(q), dev(off), 10)
        ix.sync()
    od, oj = oracle.knn(ref, q, 5)
    assert np.array_equal(idx.cpu().numpy(), oj) and np.array_equal(dist.cpu().numpy(), od)
    ot, oc = oracle.local_nbnn(ref, labels, 4, q, off, 10)
    assert np.array_equal(t.cpu().numpy(), ot) and np.array_equal(c.cpu().numpy(), oc)
