"""Pins for the CPU oracle: checks against things other than the oracle itself.

Each ``pin_*`` takes an ``oracle.Oracle`` and raises AssertionError when the
oracle disagrees with what the paper and the mathematics fix:

* library routines: scipy's ``cdist`` (squared Euclidean) and ``cKDTree``
  (exact kd-tree kNN, a different algorithm from the oracle's scan);
* exhaustive enumeration on tiny inputs with many ties;
* hand-worked cases of Alg. 1 and Alg. 2 on one-coordinate descriptors;
* closed forms: the Local NBNN totals equal sum_i min(0, NN_C(d_i) - dist_B(d_i))
  (derived from Alg. 2 for exact neighbours), the 1-class case, the
  1-descriptor case;
* location-weighted rows (130 bytes): scipy distances and kd-tree neighbours
  of the vectors with the location repeated w times, weight 0 against the
  128-byte results, and Alg. 1 / Alg. 2 totals rebuilt from those distances;
* invariants: permutation of the reference set, k + 1 = N reduces Local NBNN to
  NBNN minus a class-independent constant (Section 5.1: large k reverts to
  NBNN), the background-class discount does not move the argmin (Section 4),
  totals are never positive.

The same functions run against deliberately broken builds of the oracle in
``test_oracle_mutations.py``; every planted mistake must fail at least one.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree
from scipy.spatial.distance import cdist


def _u8(rng, n, hi=256):
    return rng.integers(0, hi, size=(n, 128), dtype=np.int64).astype(np.uint8)


def _cd(q, r):
    """Squared Euclidean distances by scipy, as exact int64."""
    return cdist(q.astype(np.float64), r.astype(np.float64), "sqeuclidean").round().astype(np.int64)


def _one_coord(values):
    """Descriptors whose only non-zero coordinate is coordinate 0."""
    a = np.zeros((len(values), 128), dtype=np.uint8)
    a[:, 0] = values
    return a


def _numpy_closed_form(ref, labels, C, q, offsets, k):
    """sum over an image's descriptors of min(0, NN_C(d) - dist_B(d)), by numpy."""
    d = _cd(q, ref)
    n_img = len(offsets) - 1
    tot = np.zeros((n_img, C), dtype=np.int64)
    for i in range(n_img):
        for row in range(offsets[i], offsets[i + 1]):
            dist_b = np.sort(d[row])[k]
            for c in range(C):
                members = d[row][labels == c]
                if members.size:
                    tot[i, c] += min(0, int(members.min()) - int(dist_b))
    return tot


def _small_case(seed, N=60, C=4, n_img=3, per_img=5, hi=256, dims=128):
    rng = np.random.default_rng(seed)
    ref = np.zeros((N, 128), dtype=np.uint8)
    q = np.zeros((n_img * per_img, 128), dtype=np.uint8)
    cols = rng.choice(128, size=dims, replace=False)
    ref[:, cols] = rng.integers(0, hi, size=(N, dims))
    q[:, cols] = rng.integers(0, hi, size=(n_img * per_img, dims))
    labels = rng.integers(0, C, size=N).astype(np.int32)
    labels[:C] = np.arange(C)  # every class present
    offsets = np.arange(0, n_img * per_img + 1, per_img, dtype=np.int64)
    return ref, labels, q, offsets


# ----------------------------------------------------------------- distance

def pin_sqdist_matches_scipy(orc):
    rng = np.random.default_rng(1)
    r, q = _u8(rng, 40), _u8(rng, 7)
    r[0], r[1], q[0], q[1] = 0, 255, 255, 0
    assert np.array_equal(orc.sqdist_matrix(r, q), _cd(q, r))


def pin_sqdist_closed_forms(orc):
    vals = [0, 1, 7, 128, 254, 255]
    a = np.array([[v] * 128 for v in vals], dtype=np.uint8)
    got = orc.sqdist_matrix(a, a)
    for i, x in enumerate(vals):
        for j, y in enumerate(vals):
            assert got[i, j] == 128 * (x - y) ** 2  # ||x*1 - y*1||^2 = 128 (x-y)^2
    q = np.zeros((1, 128), dtype=np.uint8)
    q[0, 127] = 200
    assert orc.sqdist_matrix(np.zeros((1, 128), np.uint8), q)[0, 0] == 40000
    assert orc.sqdist_matrix(np.full((1, 128), 255, np.uint8), np.zeros((1, 128), np.uint8))[0, 0] == 8323200


# ---------------------------------------------------------------------- kNN

def pin_knn_exhaustive_ties(orc):
    """N <= 8 references, 3 coordinates in {0..3}: many ties; full sort by (dist, idx)."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        N, M = int(rng.integers(1, 9)), int(rng.integers(1, 4))
        ref = np.zeros((N, 128), np.uint8)
        q = np.zeros((M, 128), np.uint8)
        cols = rng.choice(128, size=3, replace=False)
        ref[:, cols] = rng.integers(0, 4, size=(N, 3))
        q[:, cols] = rng.integers(0, 4, size=(M, 3))
        kk = int(rng.integers(1, N + 1))
        d, j = orc.knn(ref, q, kk)
        full = _cd(q, ref)
        for i in range(M):
            order = sorted(range(N), key=lambda t: (full[i, t], t))[:kk]
            assert list(j[i]) == order
            assert list(d[i]) == [full[i, t] for t in order]


def pin_knn_matches_kdtree(orc):
    rng = np.random.default_rng(3)
    r, q = _u8(rng, 600), _u8(rng, 25)
    kk = 12
    d, j = orc.knn(r, q, kk)
    td, tj = cKDTree(r.astype(np.float64)).query(q.astype(np.float64), k=kk)
    assert np.array_equal(d, np.rint(td ** 2).astype(np.int64))
    uniq = np.ones_like(d, dtype=bool)
    uniq[:, 1:] &= d[:, 1:] != d[:, :-1]
    uniq[:, :-1] &= d[:, :-1] != d[:, 1:]
    assert np.array_equal(j[uniq], tj[uniq])


def pin_knn_duplicates_and_self(orc):
    rng = np.random.default_rng(4)
    r = _u8(rng, 30)
    r[9] = r[5]
    r[17] = r[5]
    d, j = orc.knn(r, r[5:6], 4)
    assert list(d[0, :3]) == [0, 0, 0] and list(j[0, :3]) == [5, 9, 17] and d[0, 3] > 0
    # all-zero references: every distance equal, indices in order
    z = np.zeros((6, 128), np.uint8)
    d, j = orc.knn(z, _one_coord([3]), 6)
    assert list(d[0]) == [9] * 6 and list(j[0]) == list(range(6))


# --------------------------------------------------------------- Local NBNN

def pin_lnbnn_hand_worked(orc):
    """Alg. 2 by hand on one-coordinate descriptors.

    refs (value, class): r0=(0,c0) r1=(1,c1) r2=(3,c0) r3=(4,c2) r4=(10,c1).
    Image 0, k=2, descriptors 2 and 9:
      d=2: distances 4,1,1,4,64 -> order r1(1),r2(1),r0(4),... ; dist_B = 4
           c1: 1-4 = -3 ; c0: 1-4 = -3
      d=9: distances 81,64,36,25,1 -> order r4(1),r3(25),r2(36) ; dist_B = 36
           c1: 1-36 = -35 ; c2: 25-36 = -11
      totals = (-3, -38, -11) -> class 1.
    Image 1, k=2, descriptor 2 alone: totals (-3, -3, 0) -> tie, lowest class 0.
    """
    ref = _one_coord([0, 1, 3, 4, 10])
    lab = np.array([0, 1, 0, 2, 1], np.int32)
    q = _one_coord([2, 9, 2])
    t, c = orc.local_nbnn(ref, lab, 3, q, np.array([0, 2, 3]), 2)
    assert t.tolist() == [[-3, -38, -11], [-3, -3, 0]]
    assert c.tolist() == [1, 0]


def pin_lnbnn_hand_worked_repeat_class(orc):
    """k=3, refs r0=(0,c0) r1=(1,c1) r2=(3,c1) r3=(4,c2) r4=(10,c1), descriptor 2:
    order r1(1,c1) r2(1,c1) r0(4,c0) | r3(4): dist_B = 4; c1 once with min 1 -> -3;
    c0 present at distance 4 -> 4-4 = 0; c2 absent.  Descriptor 3 (k=3):
    distances 9,4,0,1,49 -> r2(0,c1) r3(1,c2) r1(4,c1) | r0(9): dist_B = 9;
    c1: 0-9 = -9, c2: 1-9 = -8."""
    ref = _one_coord([0, 1, 3, 4, 10])
    lab = np.array([0, 1, 1, 2, 1], np.int32)
    t, c = orc.local_nbnn(ref, lab, 3, _one_coord([2, 3]), np.array([0, 1, 2]), 3)
    assert t.tolist() == [[0, -3, 0], [0, -9, -8]]
    assert c.tolist() == [1, 1]


def pin_lnbnn_numpy_closed_form(orc):
    """Alg. 2 totals equal sum_i min(0, NN_C - dist_B) computed by scipy + numpy."""
    for seed, hi, dims in ((5, 256, 128), (6, 4, 3), (7, 2, 5)):
        ref, lab, q, off = _small_case(seed, hi=hi, dims=dims)
        for k in (1, 2, 5, 59):
            want = _numpy_closed_form(ref, lab, 4, q, off, k)
            t, c = orc.local_nbnn(ref, lab, 4, q, off, k)
            assert np.array_equal(t, want), (seed, k)
            assert list(c) == [int(np.argmin(row)) for row in want]
            t2, _ = orc.local_nbnn_closed_form(ref, lab, 4, q, off, k)
            assert np.array_equal(t2, want), (seed, k)


def pin_lnbnn_one_class(orc):
    """C = 1: totals[0] = sum_i (d_(1) - d_(k+1))."""
    rng = np.random.default_rng(8)
    ref, q = _u8(rng, 50), _u8(rng, 6)
    d = np.sort(_cd(q, ref), axis=1)
    for k in (1, 3, 49):
        t, c = orc.local_nbnn(ref, np.zeros(50, np.int32), 1, q, np.array([0, 6]), k)
        assert t[0, 0] == int((d[:, 0] - d[:, k]).sum()) and c[0] == 0


def pin_lnbnn_one_descriptor(orc):
    """One descriptor: totals[C] = min(0, NN_C - d_(k+1))."""
    rng = np.random.default_rng(9)
    ref, q = _u8(rng, 40), _u8(rng, 1)
    lab = (np.arange(40) % 5).astype(np.int32)
    d = _cd(q, ref)[0]
    for k in (1, 4, 10):
        dist_b = np.sort(d)[k]
        want = [min(0, int(d[lab == c].min()) - int(dist_b)) for c in range(5)]
        t, _ = orc.local_nbnn(ref, lab, 5, q, np.array([0, 1]), k)
        assert t[0].tolist() == want


def pin_lnbnn_permutation_invariant(orc):
    for seed, hi, dims in ((10, 256, 128), (11, 3, 4)):
        ref, lab, q, off = _small_case(seed, hi=hi, dims=dims)
        perm = np.random.default_rng(seed).permutation(len(ref))
        for k in (1, 3, 10):
            a, ca = orc.local_nbnn(ref, lab, 4, q, off, k)
            b, cb = orc.local_nbnn(ref[perm], lab[perm], 4, q, off, k)
            assert np.array_equal(a, b) and np.array_equal(ca, cb)


def pin_lnbnn_full_k_reduces_to_nbnn(orc):
    """k + 1 = N: Local totals = NBNN totals - sum_i dist_B(d_i), dist_B = farthest."""
    ref, lab, q, off = _small_case(12, N=30)
    far = _cd(q, ref).max(axis=1)
    loc, lc = orc.local_nbnn(ref, lab, 4, q, off, 29)
    nb, nc = orc.nbnn(ref, lab, 4, q, off)
    for i in range(len(off) - 1):
        const = int(far[off[i]:off[i + 1]].sum())
        assert (nb[i] - loc[i]).tolist() == [const] * 4
    assert np.array_equal(lc, nc)


def pin_lnbnn_background_discount(orc):
    """Section 4: giving absent classes dist_B instead of skipping them shifts every
    class by the same sum_i dist_B(d_i), so the argmin is unchanged."""
    ref, lab, q, off = _small_case(13, N=80, C=4)
    k = 4
    d, j = orc.knn(ref, q, k + 1)
    for i in range(len(off) - 1):
        full = np.zeros(4, np.int64)
        dist_b_sum = 0
        for row in range(off[i], off[i + 1]):
            dist_b = d[row, k]
            dist_b_sum += dist_b
            for c in range(4):
                present = [d[row, a] for a in range(k) if lab[j[row, a]] == c]
                full[c] += min(present) if present else dist_b
        t, cls = orc.local_nbnn(ref, lab, 4, q[off[i]:off[i + 1]], np.array([0, off[i + 1] - off[i]]), k)
        assert (full - t[0]).tolist() == [dist_b_sum] * 4
        assert cls[0] == int(np.argmin(full))


def pin_lnbnn_sign_and_support(orc):
    """Totals are <= 0 and one descriptor updates at most k classes."""
    ref, lab, q, off = _small_case(14, N=100, C=8, n_img=12, per_img=1)
    for k in (1, 2, 3):
        t, _ = orc.local_nbnn(ref, lab, 8, q, off, k)
        assert (t <= 0).all()
        assert ((t != 0).sum(axis=1) <= k).all()
        assert (t.sum(axis=1) < 0).any()


def pin_lnbnn_edge_cases(orc):
    import oracle
    ref, lab, q, off = _small_case(15, N=12)
    # an image with no descriptors: zero totals, class 0
    t, c = orc.local_nbnn(ref, lab, 4, q[:3], np.array([0, 0, 3, 3]), 2)
    assert t[0].tolist() == [0, 0, 0, 0] and t[2].tolist() == [0, 0, 0, 0]
    assert c[0] == 0 and c[2] == 0
    for bad_k in (0, 12):
        try:
            orc.local_nbnn(ref, lab, 4, q, off, bad_k)
        except oracle.OracleError as e:
            assert e.code == -3
        else:
            raise AssertionError("k out of range accepted")
    bad = lab.copy()
    bad[3] = 4
    try:
        orc.local_nbnn(ref, bad, 4, q, off, 2)
    except oracle.OracleError as e:
        assert e.code == -2
    else:
        raise AssertionError("label out of range accepted")


# -------------------------------------------------------------------- NBNN

def pin_class_min_matches_scipy(orc):
    ref, lab, q, _ = _small_case(16, N=70, C=5)
    d = _cd(q, ref)
    want = np.stack([d[:, lab == c].min(axis=1) for c in range(5)], axis=1)
    assert np.array_equal(orc.class_min(ref, lab, 5, q), want)


def pin_nbnn_hand_worked(orc):
    """Alg. 1 on the refs of ``pin_lnbnn_hand_worked``: descriptor 2 -> NN_C = (1, 1, 4),
    descriptor 9 -> (36, 1, 25); image totals (37, 2, 29) -> class 1.
    Descriptor 3 alone -> (0, 4, 1) -> class 0."""
    ref = _one_coord([0, 1, 3, 4, 10])
    lab = np.array([0, 1, 0, 2, 1], np.int32)
    t, c = orc.nbnn(ref, lab, 3, _one_coord([2, 9, 3]), np.array([0, 2, 3]))
    assert t.tolist() == [[37, 2, 29], [0, 4, 1]]
    assert c.tolist() == [1, 0]


def pin_nbnn_matches_scipy(orc):
    ref, lab, q, off = _small_case(17, N=90, C=6, n_img=4, per_img=7)
    d = _cd(q, ref)
    cm = np.stack([d[:, lab == c].min(axis=1) for c in range(6)], axis=1)
    want = np.stack([cm[off[i]:off[i + 1]].sum(axis=0) for i in range(4)])
    t, c = orc.nbnn(ref, lab, 6, q, off)
    assert np.array_equal(t, want)
    assert c.tolist() == [int(np.argmin(r)) for r in want]


def pin_nbnn_ties_and_errors(orc):
    import oracle
    rng = np.random.default_rng(18)
    half = _u8(rng, 10)
    ref = np.concatenate([half, half])
    lab = np.array([0] * 10 + [1] * 10, np.int32)
    t, c = orc.nbnn(ref, lab, 2, _u8(rng, 3), np.array([0, 3]))
    assert t[0, 0] == t[0, 1] and c[0] == 0  # tie -> lowest class
    try:
        orc.nbnn(ref, lab, 3, _u8(rng, 3), np.array([0, 3]))  # class 2 has no references
    except oracle.OracleError as e:
        assert e.code == -4
    else:
        raise AssertionError("empty class accepted")


# ------------------------------------------------------------ coarse shortlist
#
# The coarse-shortlist form is this project's approximate search (shift each
# coordinate by 64, round to FP8 E4M3, coarse = ||q'||^2 + ||r'||^2 - 2 q~.r~,
# keep the m smallest, rerank by exact distance).  Its pins: PyTorch's own
# E4M3 conversion, hand-worked values, the identity coarse == exact distance
# when no coordinate needs rounding, and the reduction to exact search when
# the shortlist holds every reference.

def _torch_e4m3(x):
    import torch
    t = torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.float8_e4m3fn)
    return t.to(torch.float32).numpy().astype(np.int64)


def pin_e4m3_matches_torch(orc):
    x = np.arange(-448, 449)
    assert np.array_equal(orc.e4m3_round(x), _torch_e4m3(x))


def pin_e4m3_hand_worked(orc):
    # below 16 every integer is exact; 36 (step 4) exact; 68 is half-way between
    # 64 and 72 -> even mantissa 64; 76 between 72 and 80 -> 80; 191 -> 192
    x = np.array([0, 7, 15, -15, 17, 36, 68, 76, 191, -64, -68, 255])
    assert orc.e4m3_round(x).tolist() == [0, 7, 15, -15, 16, 36, 64, 80, 192, -64, -64, 256]


def pin_coarse_hand_worked(orc):
    """One moving coordinate, all others 64 (shifted to 0):
    (255, 0): 191^2 + 64^2 - 2 * 192 * (-64) = 65153 (exact 65025);
    (100, 90): 36 and 26 are exact -> 10^2 = 100;
    (147, 163): 83 -> 80, 99 -> 96: 83^2 + 99^2 - 2 * 80 * 96 = 1330 (exact 256);
    (132, 140): 68 -> 64, 76 -> 80: 68^2 + 76^2 - 2 * 64 * 80 = 160 (exact 64)."""
    def one(v):
        a = np.full((1, 128), 64, np.uint8)
        a[0, 0] = v
        return a
    got = [int(orc.coarse_matrix(one(b), one(a))[0, 0]) for a, b in [(255, 0), (100, 90), (147, 163), (132, 140)]]
    assert got == [65153, 100, 1330, 160]


def pin_coarse_exact_when_representable(orc):
    # coordinates in [49, 79]: x - 64 in [-15, 15] needs no rounding, so the
    # coarse value is ||q' - r'||^2 = ||q - r||^2 exactly
    rng = np.random.default_rng(30)
    ref = rng.integers(49, 80, size=(40, 128)).astype(np.uint8)
    q = rng.integers(49, 80, size=(6, 128)).astype(np.uint8)
    assert np.array_equal(orc.coarse_matrix(ref, q), _cd(q, ref))


def pin_knn_coarse_full_shortlist_is_exact(orc):
    rng = np.random.default_rng(31)
    ref = _u8(rng, 50, hi=6)  # few values: many ties
    q = _u8(rng, 7, hi=6)
    d = _cd(q, ref)
    for kk in (1, 5, 50):
        od, oj = orc.knn_coarse(ref, q, kk, 50)
        for i in range(len(q)):
            order = np.lexsort((np.arange(50), d[i]))[:kk]
            assert oj[i].tolist() == order.tolist() and od[i].tolist() == d[i][order].tolist()
        od2, oj2 = orc.knn_coarse(ref, q, kk, 500)  # m > N: still all of them
        assert np.array_equal(oj2, oj)


def pin_knn_coarse_brute_force(orc):
    """Shortlist by sorting the whole coarse matrix (coordinates rounded by
    PyTorch), rerank by scipy distances, on 60 references."""
    rng = np.random.default_rng(32)
    ref = _u8(rng, 60)
    q = _u8(rng, 8)
    qs = _torch_e4m3(q.astype(np.int64) - 64)
    rs = _torch_e4m3(ref.astype(np.int64) - 64)
    cz = ((q.astype(np.int64) - 64) ** 2).sum(1)[:, None] + ((ref.astype(np.int64) - 64) ** 2).sum(1)[None, :] \
        - 2 * qs @ rs.T
    d = _cd(q, ref)
    for kk, m in ((3, 3), (4, 9), (10, 20)):
        od, oj = orc.knn_coarse(ref, q, kk, m)
        for i in range(len(q)):
            short = np.lexsort((np.arange(60), cz[i]))[:m]
            best = short[np.lexsort((short, d[i][short]))][:kk]
            assert oj[i].tolist() == best.tolist() and od[i].tolist() == d[i][best].tolist()


def pin_lnbnn_coarse_full_shortlist_is_exact(orc):
    ref, lab, q, off = _small_case(33, N=45, C=4, n_img=3, per_img=6)
    for k in (1, 4, 44):
        t, c = orc.local_nbnn_coarse(ref, lab, 4, q, off, k, 45)
        assert np.array_equal(t, _numpy_closed_form(ref, lab, 4, q, off, k))
        assert c.tolist() == [int(np.argmin(r)) for r in t]


def pin_lnbnn_coarse_short_list(orc):
    """With a short list the neighbours are the exact nearest of the shortlist:
    totals follow Alg. 2 on them (hand-check through knn_coarse)."""
    ref, lab, q, off = _small_case(34, N=80, C=5, n_img=2, per_img=5)
    k, m = 3, 6
    t, _ = orc.local_nbnn_coarse(ref, lab, 5, q, off, k, m)
    nd, nj = orc.knn_coarse(ref, q, k + 1, m)
    want = np.zeros_like(t)
    for i in range(2):
        for row in range(off[i], off[i + 1]):
            for c in set(lab[nj[row][:k]].tolist()):
                want[i, c] += min(int(nd[row][a]) for a in range(k) if lab[nj[row][a]] == c) - int(nd[row][k])
    assert np.array_equal(t, want)
    # the reranked distances are the exact distances of the returned rows
    d = _cd(q, ref)
    assert np.array_equal(nd, np.take_along_axis(d, nj, axis=1))


# ----------------------------------------------------------------- location

def _loc_case(seed, N, M, hi=256, loc_hi=256):
    """130-byte rows: 128 appearance bytes, then 2 location bytes."""
    rng = np.random.default_rng(seed)
    ref = rng.integers(0, hi, size=(N, 130)).astype(np.uint8)
    q = rng.integers(0, hi, size=(M, 130)).astype(np.uint8)
    ref[:, 128:] = rng.integers(0, loc_hi, size=(N, 2))
    q[:, 128:] = rng.integers(0, loc_hi, size=(M, 2))
    return ref, q


def _expanded(a, w):
    """130-byte rows as float vectors of 128 + 2w coordinates, the location
    repeated w times: their plain squared distances are the weighted ones."""
    a = np.asarray(a, dtype=np.float64)
    return np.concatenate([a[:, :128]] + [a[:, 128:130]] * w, axis=1)


def _cd_loc(q, r, w):
    return cdist(_expanded(q, w), _expanded(r, w), "sqeuclidean").round().astype(np.int64)


def pin_location_matches_scipy(orc):
    for w in (0, 1, 3, 48):
        ref, q = _loc_case(30 + w, 50, 9)
        assert np.array_equal(orc.sqdist_matrix(ref, q, location_weight=w), _cd_loc(q, ref, w)), w
    a = np.zeros((1, 130), np.uint8)
    b = a.copy()
    b[0, 129] = 200
    assert orc.sqdist_matrix(a, b, location_weight=7)[0, 0] == 7 * 40000
    b[0, :128] = 255
    assert orc.sqdist_matrix(a, b, location_weight=7)[0, 0] == 8323200 + 7 * 40000


def pin_location_knn_matches_kdtree(orc):
    ref, q = _loc_case(40, 500, 20)
    w, kk = 5, 10
    d, j = orc.knn(ref, q, kk, location_weight=w)
    td, tj = cKDTree(_expanded(ref, w)).query(_expanded(q, w), k=kk)
    assert np.array_equal(d, np.rint(td ** 2).astype(np.int64))
    uniq = np.ones_like(d, dtype=bool)
    uniq[:, 1:] &= d[:, 1:] != d[:, :-1]
    uniq[:, :-1] &= d[:, :-1] != d[:, 1:]
    assert np.array_equal(j[uniq], tj[uniq])


def pin_location_weight_zero_is_appearance(orc):
    ref, q = _loc_case(41, 80, 12)
    lab = (np.arange(80) % 4).astype(np.int32)
    off = np.array([0, 5, 12], np.int64)
    for k in (1, 5):
        a = orc.local_nbnn(ref, lab, 4, q, off, k, location_weight=0)
        b = orc.local_nbnn(ref[:, :128], lab, 4, q[:, :128], off, k)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    a = orc.nbnn(ref, lab, 4, q, off, location_weight=0)
    b = orc.nbnn(ref[:, :128], lab, 4, q[:, :128], off)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def pin_location_local_nbnn_closed_form(orc):
    """Alg. 2 and Alg. 1 under the weighted distance, from scipy distances on the
    expanded vectors: sum_i min(0, NN_C - dist_B) and sum_i NN_C; many ties."""
    ref, q = _loc_case(42, 60, 10, hi=4, loc_hi=8)
    lab = (np.arange(60) % 4).astype(np.int32)
    off = np.array([0, 4, 4, 10], np.int64)
    w = 3
    D = _cd_loc(q, ref, w)
    for k in (1, 3, 59):
        want = np.zeros((3, 4), np.int64)
        for i in range(3):
            for row in range(off[i], off[i + 1]):
                dist_b = np.sort(D[row])[k]
                for c in range(4):
                    want[i, c] += min(0, int(D[row][lab == c].min()) - int(dist_b))
        t, c = orc.local_nbnn(ref, lab, 4, q, off, k, location_weight=w)
        assert np.array_equal(t, want), k
        t2, _ = orc.local_nbnn_closed_form(ref, lab, 4, q, off, k, location_weight=w)
        assert np.array_equal(t2, want), k
    nb = np.zeros((3, 4), np.int64)
    for i in range(3):
        for row in range(off[i], off[i + 1]):
            nb[i] += [int(D[row][lab == c].min()) for c in range(4)]
    t, c = orc.nbnn(ref, lab, 4, q, off, location_weight=w)
    assert np.array_equal(t, nb)
    assert np.array_equal(orc.class_min(ref, lab, 4, q, location_weight=w),
                          np.array([[D[r][lab == c].min() for c in range(4)] for r in range(10)]))


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
