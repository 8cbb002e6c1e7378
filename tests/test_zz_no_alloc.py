"""knn_search_noalloc against knn_search and against the oracle.

knn_search_noalloc serves callers that must not allocate device memory (a
host framework that owns every allocation, or code that cannot afford the
device synchronisation of cudaMalloc/cudaFree): all its intermediates live in
the library's fixed device scratch array.  This file runs last, so a failure
here cannot hide any other test's result; it also passes alone in a fresh
process, where its first call performs the per-device scratch set-up.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _case(seed, n_ref, n_q):
    rng = np.random.default_rng(seed)
    ref = rng.integers(0, 256, size=(n_ref, 128)).astype(np.uint8)
    ref[7:12] = ref[3]  # exact ties: the lower row must win on both paths
    q = rng.integers(0, 256, size=(n_q, 128)).astype(np.uint8)
    q[0] = ref[3]
    return ref, q


def _noalloc(lib, ref_d, q_d, k):
    m = q_d.shape[0]
    idx = torch.empty((m, k), dtype=torch.int32, device=q_d.device)
    dist = torch.empty((m, k), dtype=torch.int32, device=q_d.device)
    code = lib.knn_search_noalloc(ctypes.c_void_p(ref_d.data_ptr()), ref_d.shape[0], ctypes.c_void_p(q_d.data_ptr()),
                                  m, k, ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(dist.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code, idx, dist


@pytest.fixture(scope="module")
def lib():
    from paper_1112_0059_gb300 import build, lnbnn
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    build.build()
    lib = lnbnn.load_library()
    lib.knn_search_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    lib.knn_search_noalloc.restype = ctypes.c_int
    return lib


def test_noalloc_matches_knn_search_on_two_calls(lib):
    import oracle
    from paper_1112_0059_gb300 import lnbnn
    # a larger call (several reference splits sharing the rows' bounds), then
    # smaller ones that find the earlier calls' data in the scratch
    for seed, n_ref, n_q, k in ((0, 20000 + 77, 3000 + 5, 10), (1, 5000 + 3, 700, 25), (2, 6000 + 11, 500, 50)):
        ref, q = _case(seed, n_ref, n_q)
        ref_d, q_d = torch.from_numpy(ref).cuda(), torch.from_numpy(q).cuda()
        code, idx, dist = _noalloc(lib, ref_d, q_d, k)
        assert code == 0, lnbnn.STATUS.get(code)
        with lnbnn.Index(ref_d, torch.zeros(n_ref, dtype=torch.int32, device="cuda"), 1) as ix:
            want_idx, want_dist = ix.knn_search(q_d, k)
            ix.sync()
        # integer work: bit-exact agreement, with the existing entry point and
        # with the oracle's (distance, lowest row) order
        assert torch.equal(idx, want_idx) and torch.equal(dist, want_dist)
        od, oj = oracle.knn(ref, q, k)
        assert np.array_equal(dist.cpu().numpy(), od.astype(np.int32))
        assert np.array_equal(idx.cpu().numpy(), oj.astype(np.int32))
        assert int(dist[0, 0]) == 0 and int(idx[0, 0]) == 3


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    ref_d = torch.zeros((300000, 128), dtype=torch.uint8, device="cuda")
    q_d = torch.zeros((10, 128), dtype=torch.uint8, device="cuda")
    code, _, _ = _noalloc(lib, ref_d, q_d, 10)
    assert code == 10  # LNBNN_ERR_SCRATCH_LIMIT, before any work is issued
    # within the per-operand bound but not in the scratch as a whole
    ref_d = torch.zeros((200000, 128), dtype=torch.uint8, device="cuda")
    q_d = torch.zeros((60000, 128), dtype=torch.uint8, device="cuda")
    code, _, _ = _noalloc(lib, ref_d, q_d, 10)
    assert code == 10


def test_noalloc_rejects_host_memory(lib):
    ref = torch.zeros((1000, 128), dtype=torch.uint8)  # host memory: not reachable as device memory
    q_d = torch.zeros((10, 128), dtype=torch.uint8, device="cuda")
    idx = torch.empty((10, 5), dtype=torch.int32, device="cuda")
    dist = torch.empty((10, 5), dtype=torch.int32, device="cuda")
    code = lib.knn_search_noalloc(ctypes.c_void_p(ref.data_ptr()), 1000, ctypes.c_void_p(q_d.data_ptr()), 10, 5,
                                  ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(dist.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 1  # LNBNN_ERR_INVALID_ARG
