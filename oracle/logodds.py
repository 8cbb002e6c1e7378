"""CPU oracle for NBNN as a sum of log-odds increments -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product path never does.

Paper: McCann & Lowe, "Local Naive Bayes Nearest Neighbor", Section 3.1.
Each query descriptor d changes the posterior log-odds of every class C by

    increment(d, C) = log [ P(C|d) P(Cbar) ] / [ P(Cbar|d) P(C) ]      Eq. (eqn:log-odds)

with Cbar the set of all other classes, and the image goes to the class with
the largest sum of increments (Eq. (eqn:log-increments); the prior term is
dropped for equal priors, P(C) = 1 / |classes|).  The posterior follows the
original NBNN's Gaussian kernel on the nearest neighbour of each class:

    P(C|d) = exp(-beta ||d - NN_C(d)||^2) / sum_C' exp(-beta ||d - NN_C'(d)||^2),

beta = 1 / (2 sigma^2) (Section 3, the kernel of Eq. (eqn:nbnn)).  The paper
leaves sigma unstated, so beta is an argument.  The "positive increments only"
variant (Table 1) adds an increment only where it is > 0.

Arithmetic is float64 numpy; ``scipy.special.logsumexp`` is the one library
step (log of a sum of exponentials without underflow).  The NN_C(d) distances
come from the C oracle's ``class_min``.
"""
from __future__ import annotations

import numpy as np
from scipy.special import logsumexp

from . import class_min


def logodds_increments(nn_dist, beta: float) -> np.ndarray:
    """increment[i, C] of Eq. (eqn:log-odds) from nn_dist[i, C] = ||d_i - NN_C(d_i)||^2."""
    D = np.asarray(nn_dist, dtype=np.float64)
    n_cls = D.shape[1]
    if n_cls < 2:
        raise ValueError("the log-odds need at least two classes")
    L = -float(beta) * D                                   # log of the unnormalised kernel
    log_z = logsumexp(L, axis=1)                           # log sum over all classes
    log_post = L - log_z[:, None]                          # log P(C|d)
    log_post_bar = np.empty_like(L)                        # log P(Cbar|d): the other classes
    for c in range(n_cls):
        log_post_bar[:, c] = logsumexp(np.delete(L, c, axis=1), axis=1) - log_z
    log_prior = np.log(1.0 / n_cls)                        # log P(C)
    log_prior_bar = np.log((n_cls - 1) / n_cls)            # log P(Cbar)
    return (log_post + log_prior_bar) - (log_post_bar + log_prior)


def decision_tolerance(nn_dist, beta: float) -> float:
    """|increment| below which a float64 rounding could flip its sign: the
    increments are differences of terms up to beta * max distance."""
    D = np.asarray(nn_dist, dtype=np.float64)
    return 1e-9 * (1.0 + float(beta) * (float(D.max()) if D.size else 0.0))


def sum_increments(inc, offsets, positive_only: bool, tol: float = 0.0):
    """Per-image sums of the increments (all, or only the positive ones), the
    argmax class (lowest class on ties; 0 for an empty image), the number of
    increments added per image, and the number of increments within tol of 0
    (whose inclusion a rounding could change)."""
    inc = np.asarray(inc, dtype=np.float64)
    offsets = np.asarray(offsets, dtype=np.int64)
    n_img, n_cls = len(offsets) - 1, inc.shape[1]
    totals = np.zeros((n_img, n_cls), np.float64)
    counts = np.zeros(n_img, np.int64)
    near = np.zeros(n_img, np.int64)
    for g in range(n_img):
        rows = inc[offsets[g]:offsets[g + 1]]
        use = rows > 0 if positive_only else np.ones(rows.shape, bool)
        totals[g] = np.where(use, rows, 0.0).sum(axis=0)
        counts[g] = int(use.sum())
        near[g] = int((np.abs(rows) <= tol).sum())
    classes = np.argmax(totals, axis=1).astype(np.int32)  # first maximum = lowest class
    return totals, classes, counts, near


def nbnn_logodds(ref, labels, n_classes, q, offsets, beta: float, positive_only: bool, threads=0,
                 location_weight=None):
    """Classify every image by its summed log-odds increments (Eq. (eqn:log-increments)).

    Returns (totals float64 [n_img, C], classes int32 [n_img],
    increments added int64 [n_img], increments within the decision tolerance of 0 int64 [n_img]).
    130-byte rows take a location weight, as ``class_min`` does."""
    D = class_min(ref, labels, n_classes, q, threads, location_weight)
    inc = logodds_increments(D, beta) if len(D) else np.zeros((0, n_classes))
    tol = decision_tolerance(D, beta) if len(D) else 0.0
    return sum_increments(inc, offsets, positive_only, tol)
