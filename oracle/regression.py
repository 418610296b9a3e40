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
