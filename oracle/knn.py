"""k-nearest-neighbour regression and classification through the k-th order statistic
of the distances (CPU oracle, float64).

Test infrastructure only (see the package docstring).  Sec. 5 of Beliakov,
arXiv:1104.2732, last application.  kNN regression predicts f(q) as a weighted sum of
the ordinates f_i of the k training points closest to q, with weights that decrease
with the distance d_i = ||q - x_i||.  Classification takes the majority vote of those k
points.  Instead of sorting the distances, the k points are marked by an indicator
against d_(k), the k-th order statistic of the distances, formed like the weights of
Eq. (med_reg); one reduction then gives the weighted sum.

Readings (the passage is silent on each point):
* Metric.  Euclidean.  The order statistic is taken on the squared distances, which
  share the ordering; the weights use d = sqrt(d^2).
* Ties at d_(k).  The indicator is 1 below d_(k) and 0 above.  The b points at exactly
  d_(k) share a / b each, where a = k - #(d < d_(k)), as the a / b weight at the order
  statistic in Eq. (med_reg).  So exactly k points count in total, and the result is
  the mean over every way of breaking the tie.
* Weights.  w(d) = 1 (uniform) or w(d) = 1 / (d + eps) (inverse distance, eps > 0).
  The prediction is normalised: sum rho_i w_i f_i / sum rho_i w_i.
* Vote.  Class c scores sum rho_i [label_i = c] (unweighted).  The prediction is the
  highest score, and a tie between classes goes to the smallest label.  Scores are
  exact rationals (the tie share a/b as a fraction), so whether two classes tie is
  decided exactly, not by the rounding of a float sum.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from .select import select_kth


def squared_distances(X, Q):
    """(m, n) squared Euclidean distances ||q_j - x_i||^2, summed term by term in
    float64 (no expansion into norms and a product)."""
    X = np.asarray(X, dtype=np.float64)
    Q = np.asarray(Q, dtype=np.float64)
    diff = Q[:, None, :] - X[None, :, :]
    return np.einsum("mnp,mnp->mn", diff, diff)


def squared_distances_f32(X, Q):
    """(m, n) squared distances in float32 with a fixed order of operations: for
    t = 0, 1, ..., p-1, diff = q_t - x_t, then acc = acc + diff * diff, every product and
    sum rounded to float32 (no fused multiply-add).  Which points are the k nearest is
    an integer decision taken on these floats, so a float32 path takes it on exactly
    these values."""
    X = np.asarray(X, dtype=np.float32)
    Q = np.asarray(Q, dtype=np.float32)
    acc = np.zeros((Q.shape[0], X.shape[0]), dtype=np.float32)
    for t in range(X.shape[1]):
        diff = Q[:, None, t] - X[None, :, t]
        acc = acc + diff * diff
    return acc


def indicator(d2, k):
    """rho_i for one query: 1 for d_i < d_(k), a/b for d_i = d_(k), 0 above."""
    d2 = np.asarray(d2, dtype=np.float64)
    q = float(select_kth(d2, k))
    below = d2 < q
    tie = d2 == q
    a = k - int(np.count_nonzero(below))
    b = int(np.count_nonzero(tie))
    rho = np.where(below, 1.0, 0.0)
    rho[tie] = a / b
    return rho


def weight(d, kind="uniform", eps=1e-6):
    d = np.asarray(d, dtype=np.float64)
    if kind == "uniform":
        return np.ones_like(d)
    if kind == "inverse":
        return 1.0 / (d + eps)
    raise ValueError(f"unknown weight {kind!r}")


def regress(X, f, Q, k, kind="uniform", eps=1e-6):
    """kNN regression prediction for every query row of Q (m values)."""
    return regress_d2(squared_distances(X, Q), f, k, kind, eps)


def regress_d2(D2, f, k, kind="uniform", eps=1e-6):
    """kNN regression from given squared distances D2 (m, n), in float64."""
    f = np.asarray(f, dtype=np.float64)
    D2 = np.asarray(D2, dtype=np.float64)
    out = np.empty(D2.shape[0])
    for j in range(D2.shape[0]):
        rho = indicator(D2[j], k)
        w = rho * weight(np.sqrt(D2[j]), kind, eps)
        out[j] = math.fsum((w * f).tolist()) / math.fsum(w.tolist())
    return out


def exact_votes(X, labels, Q, k, n_classes):
    """Per query, the list of n_classes vote totals sum rho_i [label_i = c] as exact
    Fractions: the points below d_(k) count 1 each, the b points at d_(k) count a/b."""
    return exact_votes_d2(squared_distances(X, Q), labels, k, n_classes)


def exact_votes_d2(D2, labels, k, n_classes):
    """exact_votes from given squared distances D2 (m, n)."""
    labels = np.asarray(labels)
    D2 = np.asarray(D2, dtype=np.float64)
    out = []
    for j in range(D2.shape[0]):
        q = float(select_kth(D2[j], k))
        below = D2[j] < q
        tie = D2[j] == q
        share = Fraction(k - int(np.count_nonzero(below)), int(np.count_nonzero(tie)))
        out.append([int(np.count_nonzero(below & (labels == c))) + share * int(np.count_nonzero(tie & (labels == c)))
                    for c in range(n_classes)])
    return out


def votes(X, labels, Q, k, n_classes):
    """(m, n_classes) vote totals as floats (each the rounding of its exact value)."""
    return np.array([[float(v) for v in row] for row in exact_votes(X, labels, Q, k, n_classes)])


def classify(X, labels, Q, k, n_classes):
    """Majority class among the k nearest: the highest exact vote total, a tie between
    classes going to the smallest label."""
    return classify_d2(squared_distances(X, Q), labels, k, n_classes)


def classify_d2(D2, labels, k, n_classes):
    """classify from given squared distances D2 (m, n)."""
    out = []
    for row in exact_votes_d2(D2, labels, k, n_classes):
        out.append(row.index(max(row)))
    return np.array(out, dtype=np.int64)
