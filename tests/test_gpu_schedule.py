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
        assert tuned["runs"] >= 20 and tuned["tile_ms"] > 0, tuned
        # the large-batch forms of the exact scan were timed (no FP8 operand here)
        assert tuned["form_runs"] == 4 and all(x > 0 for x in tuned["form_ms"][:4]), tuned
        assert tuned["exact_query_tiles"] in (1, 2) and tuned["exact_persistent"] in (0, 1), tuned
        assert tuned["coarse_persistent"] == -1 and not any(tuned["form_ms"][4:]), tuned
        big = ix.plan_search(100_000, 11)
        assert (big["tile_m"], big["persistent"]) == (128 * tuned["exact_query_tiles"], tuned["exact_persistent"])
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


def _case(seed, N, M, C, hi=256):
    rng = np.random.default_rng(seed)
    ref = rng.integers(0, hi, size=(N, 128), dtype=np.uint8)
    ref[50:60] = ref[5]  # exact ties across reference tiles
    q = rng.integers(0, hi, size=(M, 128), dtype=np.uint8)
    q[:3] = ref[5]
    labels = (rng.integers(0, C, size=N)).astype(np.int32)
    labels[:C] = np.arange(C)
    cuts = np.sort(rng.integers(0, M + 1, size=6))
    offsets = np.concatenate([[0], cuts, [M]]).astype(np.int64)
    return ref, labels, q, offsets


SCHEDULES = [dict(splits=s, query_tiles=qt, persistent=p, bound_per_tile=b)
             for s in (1, 3, 8) for qt in (1, 2) for p in (0, 1) for b in (0, 1)]


def test_every_schedule_is_bit_identical(lnbnn):
    """Tile shape (one or two query tiles per CTA), grid form (one CTA per work
    item or a persistent grid with a work queue), row-bound mode and split
    count change speed only: kNN lists of every list kind, Local NBNN, NBNN
    and the FP8 shortlist all equal the oracle under each schedule."""
    N, M, C = 60_000 + 77, 3_000 + 13, 7  # 24 query tiles (an odd count of pairs is padded), ragged tails
    ref, labels, q, off = _case(90, N, M, C)
    ks = (10, 40, 100)  # register lists, 64-entry lists (one query tile per CTA only), heaps
    want = {k1: oracle.knn(ref, q, k1) for k1 in ks}
    wl = oracle.local_nbnn(ref, labels, C, q, off, 10)
    wn = oracle.nbnn(ref, labels, C, q, off)
    wf = oracle.knn_coarse(ref, q, 11, 32)
    with lnbnn.Index(dev(ref), dev(labels), C) as ix:
        ix.prepare_fp8()
        qd, od = dev(q), dev(off)
        seen = set()
        for sch in SCHEDULES:
            ix.set_schedule(**sch)
            for k1 in ks:
                plan = ix.plan_search(M, k1)
                seen.add((plan["tile_m"], plan["persistent"], plan["bound_per_tile"], k1 > 32 and k1 <= 64))
                i, d = ix.knn_search(qd, k1)
                ix.sync()
                assert np.array_equal(d.cpu().numpy(), want[k1][0]), (sch, k1)
                assert np.array_equal(i.cpu().numpy(), want[k1][1]), (sch, k1)
            t, c = ix.lnbnn_classify(qd, od, 10)
            nt, nc = ix.nbnn_classify(qd, od)
            fi, fd = ix.knn_search(qd, 11, shortlist=32)
            ix.sync()
            assert np.array_equal(t.cpu().numpy(), wl[0]) and np.array_equal(c.cpu().numpy(), wl[1]), sch
            assert np.array_equal(nt.cpu().numpy(), wn[0]) and np.array_equal(nc.cpu().numpy(), wn[1]), sch
            assert np.array_equal(fd.cpu().numpy(), wf[0]) and np.array_equal(fi.cpu().numpy(), wf[1]), sch
        ix.set_schedule(automatic=True)
    # both tile shapes, both grid forms and both bound modes were exercised
    assert {s[0] for s in seen} == {128, 256} and {s[1] for s in seen} == {0, 1}
    assert {s[2] for s in seen} >= {0, 1}


def test_schedule_arguments_are_checked(lnbnn):
    rng = np.random.default_rng(91)
    ref = rng.integers(0, 256, size=(5000, 128), dtype=np.uint8)
    with lnbnn.Index(dev(ref), dev(np.zeros(5000, np.int32)), 1) as ix:
        for bad in (dict(splits=-1), dict(query_tiles=3), dict(persistent=2), dict(bound_per_tile=-2),
                    dict(splits=100000)):
            with pytest.raises(lnbnn.LnbnnError):
                ix.set_schedule(**bad)
        ix.set_schedule(query_tiles=2, persistent=1)
        p = ix.plan_search(40_000, 11)
        assert p["tile_m"] == 256 and p["tile_n"] == 128 and p["persistent"] == 1
        p = ix.plan_search(40_000, 50)  # 64-entry lists: one query tile per CTA whatever is asked
        assert p["tile_m"] == 128 and p["tile_n"] == 256
        ix.set_schedule(automatic=True)
        p = ix.plan_search(100, 11)  # one query tile: the claimed-chunk form
        assert p["tile_m"] == 128 and p["persistent"] == 1 and p["chunked"] == 1
        assert 1 <= p["splits"] <= 5  # CTAs sharing the tile: at most one per four of the 20 reference tiles
        assert ix.plan_search(100, 51)["chunked"] == 0  # 64-entry shared-memory lists keep their splits


def test_lists_seeded_from_earlier_splits(lnbnn):
    """More query tiles than SMs and several splits run one after another: a
    split's lists start from the same rows' finished lists of the previous
    split (duplicates merged away).  Every list kind, Local NBNN and the FP8
    shortlist equal the oracle, with one CTA per item and persistent."""
    N, M, C = 30_000 + 5, 160 * 128 + 77, 6  # 161 query tiles
    ref, labels, q, off = _case(93, N, M, C)
    rows = np.random.default_rng(94).choice(M, size=1500, replace=False)
    with lnbnn.Index(dev(ref), dev(labels), C) as ix:
        ix.prepare_fp8()
        qd, od = dev(q), dev(off)
        for persistent in (0, 1):
            ix.set_schedule(splits=5, query_tiles=1, persistent=persistent, bound_per_tile=0)
            for k1 in (11, 24, 32, 101):
                i, d = ix.knn_search(qd, k1)
                ix.sync()
                od_, oj = oracle.knn(ref, q[rows], k1)
                assert np.array_equal(d.cpu().numpy()[rows], od_) and np.array_equal(i.cpu().numpy()[rows], oj), k1
            t, c = ix.lnbnn_classify(qd, od, 10)
            ix.sync()
            wt, wc = oracle.local_nbnn(ref, labels, C, q, off, 10)
            assert np.array_equal(t.cpu().numpy(), wt) and np.array_equal(c.cpu().numpy(), wc)
            ix.set_schedule(splits=5, query_tiles=2, persistent=persistent, bound_per_tile=0)
            fi, fd = ix.knn_search(qd, 11, shortlist=24)
            ix.sync()
            cd, cj = oracle.knn_coarse(ref, q[rows], 11, 24)
            assert np.array_equal(fd.cpu().numpy()[rows], cd) and np.array_equal(fi.cpu().numpy()[rows], cj)
        ix.set_schedule(automatic=True)


def test_claimed_chunks_for_few_query_tiles(lnbnn):
    """Fewer query tiles than SMs: P / T CTAs per query tile each keep its lists
    for the whole launch and claim short reference chunks in increasing order
    from a shared counter.  On a class-sorted index whose query class sits in
    one stretch of references, every list kind that takes this form (16-, 24-
    and 32-entry register lists, heaps) and the FP8 shortlist equal the
    oracle, and a fixed split count (the split form) gives the same bits."""
    rng = np.random.default_rng(101)
    C, per = 10, 30000
    N = C * per + 13
    protos = rng.integers(0, 256, size=(C, 128))
    labels = np.minimum(np.arange(N) // per, C - 1).astype(np.int32)
    ref = np.clip(protos[labels] + rng.normal(0, 20, size=(N, 128)), 0, 255).astype(np.uint8)
    ref[[40, 70000, 150000, N - 1]] = ref[7]  # exact ties in different chunks
    q = np.clip(protos[3] + rng.normal(0, 20, size=(120, 128)), 0, 255).astype(np.uint8)  # one query tile
    q[0] = ref[7]
    with lnbnn.Index(dev(ref), dev(labels), C) as ix:
        ix.prepare_fp8()
        qd = dev(q)
        for k1 in (11, 24, 32, 101):
            plan = ix.plan_search(len(q), k1)
            assert plan["chunked"] == 1 and plan["persistent"] == 1 and plan["splits"] > 1, plan
            i, d = ix.knn_search(qd, k1)
            ix.sync()
            od, oj = oracle.knn(ref, q, k1)
            assert np.array_equal(d.cpu().numpy(), od) and np.array_equal(i.cpu().numpy(), oj), k1
            ix.set_schedule(splits=3)  # the split form
            assert ix.plan_search(len(q), k1)["chunked"] == 0
            i2, d2 = ix.knn_search(qd, k1)
            ix.sync()
            assert torch.equal(i, i2) and torch.equal(d, d2), k1
            ix.set_schedule(automatic=True)
        assert ix.plan_search(len(q), 24, fp8=True)["chunked"] == 1
        fi, fd = ix.knn_search(qd, 11, shortlist=24)
        ix.sync()
        cd, cj = oracle.knn_coarse(ref, q, 11, 24)
        assert np.array_equal(fd.cpu().numpy(), cd) and np.array_equal(fi.cpu().numpy(), cj)
        q3 = np.concatenate([q, q[::-1], q[:60]])  # three query tiles: the FP8 pass still claims chunks
        assert ix.plan_search(len(q3), 24, fp8=True)["chunked"] == 1
        assert ix.plan_search(len(q3), 11)["chunked"] == 0
        f3, d3 = ix.knn_search(dev(q3), 11, shortlist=24)
        ix.sync()
        cd3, cj3 = oracle.knn_coarse(ref, q3, 11, 24)
        assert np.array_equal(d3.cpu().numpy(), cd3) and np.array_equal(f3.cpu().numpy(), cj3)
        t, c = ix.lnbnn_classify(qd, dev(np.array([0, 50, 120], dtype=np.int64)), 10)
        ix.sync()
        wt, wc = oracle.local_nbnn(ref, labels, C, q, np.array([0, 50, 120]), 10)
        assert np.array_equal(t.cpu().numpy(), wt) and np.array_equal(c.cpu().numpy(), wc)
