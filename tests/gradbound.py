"""Per-element tolerance for a float32 evaluation of the bracket network's loss
gradient (test helper, CPU only).

Each gradient element is a batch sum g_j = sum_b c_bj of per-row contributions (the
loss derivative of row b times an activation, through the backward chain).  The GPU
forms every c_bj in float32 and sums them in float32, so its error is at most
    |dg_j| <= (B u + e) * A_j,   A_j = sum_b |c_bj|,   u = 2^-24,
where B u bounds the rounding of the batch sum (a sum of B terms, any order) and e
bounds the relative rounding of one row's contribution through the forward and
backward chains.  e = 1e-4 leaves a wide margin over what float32 chains of fan-in 36,
64 and 64 actually show (a few 1e-7 relative, see tests/test_gradbound.py), yet a
mis-indexed row or column or a dropped term moves an element by a sizeable part of A_j
and is caught.  A_j is formed from the float64 oracle's own activations.  The labels are
kept away from the loss's kinks (|z - c| and ||z - c| - exp(omega)| at least 0.05), where
float32 and float64 could take different subgradient branches.
"""
from __future__ import annotations

import numpy as np

from oracle import bracket as ob

U32 = 2.0 ** -24
ROW_REL = 1e-4
KINK_MARGIN = 0.05


def kink_free_labels(theta, F, rng, z, margin=KINK_MARGIN):
    """Labels z moved away from the loss's kinks: |z - c| and ||z - c| - exp(omega)| both
    at least `margin` for the float64 network outputs (c, omega) of every row, so that a
    float32 forward pass takes the same branch of the subgradient as float64 and the
    relative rounding of z - c stays small."""
    o, _ = ob.forward(theta, F)
    c, w = o[:, 0], np.exp(o[:, 1])
    z = np.array(z, dtype=np.float64)
    for _ in range(100):
        d = z - c
        bad = (np.abs(d) < margin) | (np.abs(np.abs(d) - w) < margin)
        if not bad.any():
            return z.astype(np.float32)
        z[bad] = c[bad] + rng.normal(size=int(bad.sum())) * (1.0 + w[bad])
        z = z.astype(np.float32).astype(np.float64)
    raise RuntimeError("could not place the labels away from the kinks")


def magnitudes(theta, F, z, tau=ob.TAU):
    """A_j = sum over the batch rows of |c_bj|, the absolute per-row contributions to
    each gradient element (packed parameter order)."""
    Wf1, b1, Wf2, b2, Wf3, b3 = ob.unpack(theta)
    o, (F, u1, h1, u2, h2) = ob.forward(theta, F)
    g_o = ob.loss_grad_o(o, z, tau)
    g_u2 = (g_o @ Wf3) * ob.gelu_grad(u2)
    g_u1 = (g_u2 @ Wf2) * ob.gelu_grad(u1)
    a1, a2, ao = np.abs(g_u1), np.abs(g_u2), np.abs(g_o)
    return ob.pack([a1.T @ np.abs(F), a1.sum(axis=0), a2.T @ np.abs(h1), a2.sum(axis=0),
                    ao.T @ np.abs(h2), ao.sum(axis=0)])


def gradient_bound(theta, F, z):
    """(B u + e) * A_j: the most a float32 evaluation may differ from the float64 gradient."""
    B = np.atleast_2d(F).shape[0]
    return (B * U32 + ROW_REL) * magnitudes(theta, F, z)


def adam_first_step_bound(g64, gbound, w1_64, lr, eps=1e-8):
    """Bound on |w1_gpu - w1_64| after the first Adam step from zero moments, whose update
    is lr * phi(g) with phi(g) = g / (|g| + eps) up to the bias corrections.  phi changes
    by at most eps |dg| / ((|g| - |dg| + eps)(|g| + eps)) when |dg| < |g|, and by at most 2
    otherwise; the float32 update itself rounds by a few ulps of lr and of w1."""
    g = np.abs(g64)
    dphi = np.where(gbound < g, eps * gbound / ((g - gbound + eps) * (g + eps)), 2.0)
    return lr * (dphi + 16 * U32) + 2 * U32 * np.abs(w1_64)
