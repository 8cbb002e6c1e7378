"""Workspaces: calls that allocate nothing run concurrently on several streams
and replay from a captured CUDA graph, with results identical to the oracle."""
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


def case(seed, N, M, C, n_img=4):
    rng = np.random.default_rng(seed)
    ref = rng.integers(0, 256, size=(N, 128)).astype(np.uint8)
    q = rng.integers(0, 256, size=(M, 128)).astype(np.uint8)
    labels = (np.arange(N) % C).astype(np.int32)
    cuts = np.sort(rng.integers(0, M + 1, size=n_img - 1))
    off = np.concatenate([[0], cuts, [M]]).astype(np.int64)
    return ref, labels, q, off


def test_workspace_matches_oracle_and_limits(lnbnn):
    ref, labels, q, off = case(1, 7000, 900, 5)
    with lnbnn.Index(dev(ref), dev(labels), 5) as ix, ix.workspace(1000, 12) as ws:
        qd, od = dev(q), dev(off)
        lt, lc = ix.lnbnn_classify(qd, od, 10, workspace=ws)
        nt, nc = ix.nbnn_classify(qd, od, workspace=ws)
        idx, dist = ix.knn_search(qd, 12, workspace=ws)
        ix.sync()
        ot, oc = oracle.local_nbnn(ref, labels, 5, q, off, 10)
        assert np.array_equal(lt.cpu().numpy(), ot) and np.array_equal(lc.cpu().numpy(), oc)
        ont, onc = oracle.nbnn(ref, labels, 5, q, off)
        assert np.array_equal(nt.cpu().numpy(), ont) and np.array_equal(nc.cpu().numpy(), onc)
        od_, oj = oracle.knn(ref, q, 12)
        assert np.array_equal(dist.cpu().numpy(), od_) and np.array_equal(idx.cpu().numpy(), oj)
        big = dev(np.zeros((1200, 128), np.uint8))  # more queries than the workspace holds
        with pytest.raises(lnbnn.LnbnnError) as e:
            ix.knn_search(big, 12, workspace=ws)
        assert e.value.code == 10


def test_concurrent_streams(lnbnn):
    ref, labels, _, _ = case(2, 20000, 10, 7)
    batches = [case(10 + i, 20000, 300 + 97 * i, 7)[2:] for i in range(3)]
    with lnbnn.Index(dev(ref), dev(labels), 7) as ix:
        wss = [ix.workspace(700, 10) for _ in batches]
        streams = [torch.cuda.Stream() for _ in batches]
        outs = []
        torch.cuda.synchronize()
        for (q, off), ws, st in zip(batches, wss, streams):
            with torch.cuda.stream(st):
                outs.append(ix.lnbnn_classify(dev(q), dev(off), 10, workspace=ws, stream=st))
        torch.cuda.synchronize()
        ix.sync()
        for (q, off), (t, c) in zip(batches, outs):
            ot, oc = oracle.local_nbnn(ref, labels, 7, q, off, 10)
            assert np.array_equal(t.cpu().numpy(), ot) and np.array_equal(c.cpu().numpy(), oc)
        for ws in wss:
            ws.close()


def test_cuda_graph_replay(lnbnn):
    ref, labels, q0, off = case(3, 9000, 640, 6)
    _, _, q1, _ = case(4, 9000, 640, 6)
    with lnbnn.Index(dev(ref), dev(labels), 6) as ix, ix.workspace(640, 10) as ws:
        q_static, off_static = dev(q0), dev(off)
        tot = torch.empty((len(off) - 1, 6), dtype=torch.int64, device="cuda")
        cls = torch.empty((len(off) - 1,), dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):  # warm up outside capture
            ix.lnbnn_classify(q_static, off_static, 10, out=(tot, cls), workspace=ws)
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ix.lnbnn_classify(q_static, off_static, 10, out=(tot, cls), workspace=ws)
        for q in (q1, q0):
            q_static.copy_(dev(q))
            g.replay()
            torch.cuda.synchronize()
            ix.sync()
            ot, oc = oracle.local_nbnn(ref, labels, 6, q, off, 10)
            assert np.array_equal(tot.cpu().numpy(), ot) and np.array_equal(cls.cpu().numpy(), oc)
