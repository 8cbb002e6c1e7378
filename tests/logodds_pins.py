"""Pins for the oracle of NBNN as a sum of log-odds increments (Section 3.1).

Each ``pin_*`` takes a module with ``logodds_increments``, ``sum_increments``
and ``nbnn_logodds`` (the oracle, or a copy with a planted mistake) and raises
AssertionError where it disagrees with what the paper and the mathematics fix:

* exact rational arithmetic: with beta = ln 2 and integer distances every
  kernel value is a power of two, so each increment is the logarithm of a
  rational number computed with ``fractions.Fraction``;
* closed forms: beta = 0 (every posterior equals the prior: all increments 0);
  two classes (increment = -beta (D_C - D_other)); a far-apart case at
  beta = 1 where a naive exponential underflows;
* the sign rule: an increment is positive exactly where the posterior P(C|d)
  exceeds the prior 1/|classes| (direct softmax at moderate beta);
* the small-beta limit: to first order in beta the full sum of increments is
  beta / (|classes| - 1) (sum_C' S - |classes| S_C), S_C the NBNN sum of
  Alg. 1, so the log-odds rule then picks the NBNN class (checked against the
  C oracle's Alg. 1);
* per-image sums: an image classified alone gives the same totals as in a
  batch; the full rule adds |classes| increments per descriptor.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np


def _rng_dist(seed, m, c, hi):
    return np.random.default_rng(seed).integers(0, hi, size=(m, c)).astype(np.int64)


def pin_exact_rationals(mod):
    D = _rng_dist(1, 24, 5, 7)
    got = mod.logodds_increments(D, math.log(2.0))
    C = D.shape[1]
    for i in range(D.shape[0]):
        w = [Fraction(1, 2 ** int(d)) for d in D[i]]
        for c in range(C):
            others = sum(w[:c] + w[c + 1:], Fraction(0))
            ratio = w[c] * (C - 1) / others   # P(C|d) P(Cbar) / (P(Cbar|d) P(C))
            want = math.log(ratio.numerator) - math.log(ratio.denominator)
            assert abs(got[i, c] - want) < 1e-12, (i, c, got[i, c], want)


def pin_beta_zero(mod):
    D = _rng_dist(2, 30, 6, 100000)
    inc = mod.logodds_increments(D, 0.0)
    assert np.abs(inc).max() < 1e-12, np.abs(inc).max()
    off = np.array([0, 10, 10, 30])
    totals, classes, counts, _ = mod.sum_increments(inc, off, True)
    assert (counts == 0).all() and (classes == 0).all() and (totals == 0).all(), (counts, classes)


def pin_two_classes(mod):
    D = _rng_dist(3, 40, 2, 3000)
    for beta in (1e-4, 3e-3):
        inc = mod.logodds_increments(D, beta)
        want = -beta * (D[:, 0] - D[:, 1]).astype(np.float64)
        assert np.allclose(inc[:, 0], want, rtol=1e-9, atol=1e-12)
        assert np.allclose(inc[:, 1], -want, rtol=1e-9, atol=1e-12)


def pin_far_apart(mod):
    # beta = 1 and distances 5000 apart: exp(-5000) underflows in float64
    D = np.array([[0, 5000, 5000], [7000, 2000, 2000], [10, 10, 90000]], np.int64)
    inc = mod.logodds_increments(D, 1.0)
    l2 = math.log(2.0)
    want = np.array([[5000.0, -5000.0 + l2, -5000.0 + l2],
                     [-5000.0, l2, l2],                 # two tied nearest classes: P = 1/2 each
                     [l2, l2, -89990.0]])
    assert np.allclose(inc, want, rtol=0, atol=1e-9), inc


def pin_sign_is_posterior_above_prior(mod):
    D = _rng_dist(4, 200, 7, 4000)
    beta = 1e-3
    inc = mod.logodds_increments(D, beta)
    e = np.exp(-beta * D.astype(np.float64))
    post = e / e.sum(axis=1, keepdims=True)
    margin = np.abs(post - 1.0 / D.shape[1])
    clear = margin > 1e-9
    assert clear.mean() > 0.99
    assert np.array_equal((inc > 0)[clear], (post > 1.0 / D.shape[1])[clear])


def _case(seed, N=90, C=5, sizes=(6, 0, 9, 4)):
    rng = np.random.default_rng(seed)
    ref = rng.integers(0, 256, size=(N, 128)).astype(np.uint8)
    labels = (np.arange(N) % C).astype(np.int32)
    q = rng.integers(0, 256, size=(sum(sizes), 128)).astype(np.uint8)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return ref, labels, C, q, off


def pin_small_beta_is_nbnn(mod):
    import oracle
    ref, labels, C, q, off = _case(5)
    beta = 1e-11  # second-order terms ~ beta^2 var(D) stay below 1e-5 of the first
    totals, classes, counts, _ = mod.nbnn_logodds(ref, labels, C, q, off, beta, False)
    s_nbnn, c_nbnn = oracle.nbnn(ref, labels, C, q, off)
    for g in range(len(off) - 1):
        if off[g + 1] == off[g]:
            assert (totals[g] == 0).all() and classes[g] == 0 and counts[g] == 0
            continue
        first_order = beta / (C - 1) * (s_nbnn[g].sum() - C * s_nbnn[g].astype(np.float64))
        assert np.allclose(totals[g], first_order, rtol=1e-4, atol=0), (totals[g], first_order)
        srt = np.sort(s_nbnn[g])
        if srt[1] - srt[0] > 0:
            assert classes[g] == c_nbnn[g], (g, classes[g], c_nbnn[g])
        assert counts[g] == (off[g + 1] - off[g]) * C


def pin_images_alone(mod):
    ref, labels, C, q, off = _case(6)
    for positive_only in (False, True):
        totals, classes, counts, _ = mod.nbnn_logodds(ref, labels, C, q, off, 2e-5, positive_only)
        for g in range(len(off) - 1):
            qi = q[off[g]:off[g + 1]]
            t1, c1, n1, _ = mod.nbnn_logodds(ref, labels, C, qi, np.array([0, len(qi)]), 2e-5, positive_only)
            assert np.array_equal(t1[0], totals[g]) and c1[0] == classes[g] and n1[0] == counts[g], g
        if positive_only:
            assert (counts[off[1:] > off[:-1]] < (np.diff(off) * C)[off[1:] > off[:-1]]).all()
        else:
            assert np.array_equal(counts, np.diff(off) * C)


ALL_PINS = [pin_exact_rationals, pin_beta_zero, pin_two_classes, pin_far_apart,
            pin_sign_is_posterior_above_prior, pin_small_beta_is_nbnn, pin_images_alone]
