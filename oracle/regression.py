"""LMS and LTS objectives of high-breakdown regression (CPU oracle, float64).

Test infrastructure only (see the package docstring).  Sec. 5 of Beliakov,
arXiv:1104.2732 (the linear model, Eq. (model); the LMS and LTS objectives; the
rho-weighted form Eq. (med_reg)).

Readings:
* LMS.  "Med(r_i)^2" is read as the order statistic s_(k) of the squared residuals
  s_i = r_i^2 with k = [(n+1)/2]; it equals Med(|r|)^2.
* LTS.  h is a parameter (the paper prints both [(n+p)/2] and [(n+1)/2]); the
  objective is the sum of the h smallest s_i.
* rho weights compare s_i with q = s_(h) (the paper compares |r|^2 with Med(r)).
"""
from __future__ import annotations

import math

import numpy as np

from .select import select_kth


def residuals(X, y, theta):
    """r = y - X theta for every candidate column of theta (Eq. (model)), in float64.

    X is (n, p), y is (n,), theta is (p, C); float32 inputs are promoted exactly.
    The sign convention y - X theta only flips r, which the squares discard.
    """
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    if theta.ndim == 1:
        theta = theta[:, None]
    return y[:, None] - X @ theta


def lms(s, k):
    """LMS objective s_(k) of one vector of squared residuals (Sec. 5)."""
    return float(select_kth(np.asarray(s, dtype=np.float64), k))


def lts(s, h):
    """LTS objective: sum of the h smallest squared residuals (Sec. 5)."""
    s = np.sort(np.asarray(s, dtype=np.float64))
    return math.fsum(s[:h].tolist())


def lts_rho_form(s, h):
    """LTS through one order statistic, Eq. (med_reg): weights 1 below q = s_(h),
    a/b at q, 0 above, with b_L = #(s < q), b = #(s = q) and a = h - b_L."""
    s = np.asarray(s, dtype=np.float64)
    q = float(select_kth(s, h))
    below = s[s < q]
    b_L = below.size
    a = h - b_L
    return math.fsum(below.tolist()) + a * q


def lms_lts(X, y, theta, k, h):
    """(LMS_c, LTS_c) for every candidate c (columns of theta), float64."""
    r = residuals(X, y, theta)
    s = r * r
    C = s.shape[1]
    out_lms = np.empty(C)
    out_lts = np.empty(C)
    for c in range(C):
        out_lms[c] = lms(s[:, c], k)
        out_lts[c] = lts(s[:, c], h)
    return out_lms, out_lts


# ---------------------------------------------------------------------------------
# The estimator search (Sec. 5: computing the LMS or LTS estimator takes many
# evaluations of F(theta)).  Readings, the paper being silent on the search itself:
# * Candidates are given (elemental fits); LMS picks the candidate of least objective.
# * LTS refines the n_refine best candidates by concentration steps (C-steps): refit
#   the model by least squares on the h observations the objective retains -- the rows
#   weighted by the rho of Eq. (med_reg), 1 below q = s_(h), a/b at q, 0 above -- and
#   repeat while the objective decreases.  The objective cannot increase: the h smallest
#   squares at the new fit sum to at most the rho-weighted sum there (any weights in
#   [0, 1] of total h), which the least-squares fit makes at most the old objective.
# * Which rows are retained is an integer decision taken on float32 squared residuals,
#   so they are formed in a stated float32 order, no fused multiply-add: for
#   j = 0..p-1, acc = acc + x_j * theta_j (each product and sum rounded), r = y - acc,
#   s = r * r.  Coefficients are float32 (as the candidates): each refit is solved in
#   float64 and rounded to float32.  Objectives are float64 sums of those float32 s.
# ---------------------------------------------------------------------------------

def squared_residuals_f32(X, y, theta):
    """(n,) float32 squared residuals of one float32 coefficient vector in the stated
    order above."""
    X = np.asarray(X, dtype=np.float32)
    y = np.asarray(y, dtype=np.float32)
    theta = np.asarray(theta, dtype=np.float32).ravel()
    acc = np.zeros(X.shape[0], dtype=np.float32)
    for j in range(X.shape[1]):
        acc = acc + X[:, j] * theta[j]
    r = y - acc
    return r * r


def rho_weights(s, h):
    """The weights of Eq. (med_reg) on squared residuals s: 1 below q = s_(h), a/b at q
    (b = #(s = q), a = h - #(s < q)), 0 above; they sum to h."""
    s = np.asarray(s, dtype=np.float64)
    q = float(select_kth(s, h))
    below = s < q
    tie = s == q
    a = h - int(np.count_nonzero(below))
    b = int(np.count_nonzero(tie))
    rho = np.where(below, 1.0, 0.0)
    rho[tie] = a / b
    return rho


def c_step(X, y, theta, h):
    """One concentration step from the float32 coefficients theta: the weighted least
    squares fit sum_i rho_i (y_i - x_i . theta')^2 -> min, solved in float64 through the
    normal equations (numpy.linalg.solve) and rounded to float32."""
    s = squared_residuals_f32(X, y, theta)
    rho = rho_weights(s, h)
    Xd = np.asarray(X, dtype=np.float64)
    yd = np.asarray(y, dtype=np.float64)
    A = Xd.T @ (rho[:, None] * Xd)
    b = Xd.T @ (rho * yd)
    return np.linalg.solve(A, b).astype(np.float32)


def lts_objective_f32(X, y, theta, h):
    """LTS objective of float32 coefficients: the rho form of Eq. (med_reg) over the
    stated float32 squared residuals, summed exactly (math.fsum) in float64."""
    s = squared_residuals_f32(X, y, theta).astype(np.float64)
    q = float(select_kth(s, h))
    below = s[s < q]
    return math.fsum(below.tolist()) + (h - below.size) * q


def c_steps(X, y, theta, h, max_steps):
    """C-steps from theta while the objective decreases, at most max_steps refits.
    Returns (theta, objective, refits kept)."""
    theta = np.asarray(theta, dtype=np.float32).ravel()
    F = lts_objective_f32(X, y, theta, h)
    kept = 0
    for _ in range(max_steps):
        nxt = c_step(X, y, theta, h)
        Fn = lts_objective_f32(X, y, nxt, h)
        if not Fn < F:
            break
        theta, F = nxt, Fn
        kept += 1
    return theta, F, kept


def lms_search(X, y, thetas, k):
    """The candidate of least LMS objective (float64 residuals), the smallest index on
    ties: (index, objective).  thetas is (C, p)."""
    thetas = np.asarray(thetas)
    vals = np.array([lms((residuals(X, y, t) ** 2)[:, 0], k) for t in thetas])
    c = int(np.argmin(vals))
    return c, float(vals[c])


def lts_search(X, y, thetas, h, n_refine, max_steps):
    """The LTS estimate: the n_refine candidates of least LTS objective (float64
    residuals; smaller index first on ties), each refined by c_steps; the refined fit of
    least objective (earlier rank on ties).  Returns (theta, objective, the refined
    candidates' indices in rank order)."""
    thetas = np.asarray(thetas)
    vals = np.array([lts((residuals(X, y, t) ** 2)[:, 0], h) for t in thetas])
    order = sorted(range(len(vals)), key=lambda c: (vals[c], c))[:n_refine]
    best = None
    for c in order:
        th, F, _ = c_steps(X, y, thetas[c], h, max_steps)
        if best is None or F < best[1]:
            best = (th, F)
    return best[0], best[1], order
