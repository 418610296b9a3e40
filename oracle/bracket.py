"""Sketch features and the bracket-proposal MLP (CPU oracle, float64).

Test infrastructure only (see the package docstring).  The paper has no learned
component: this restates the network that proposes a starting bracket for
Algorithm 1 (Sec. 3) so that the GPU forward, backward and Adam kernels can be
checked against plain float64 arithmetic.  The proposal never decides a result:
the first pass checks it by counts and the cutting plane falls back to the data's
extremes (Sec. 3, step 0) for any side that fails.

Definitions (fixed here, since the paper is silent):
* Sketch.  s_j = x[j * floor(n/1024)], j = 0..1023; sorted ascending.
  mu, sd = mean and population standard deviation of the sample (sd = 1 if 0).
* Features (36): (s_(16+32i) - mu)/sd for i = 0..31, asinh((min s - mu)/sd),
  asinh((max s - mu)/sd), asinh(mu/sd), log(sd)/16.
* Network: 36 -> 64 -> 64 -> 2, GELU(u) = u * Phi(u) on both hidden layers, linear
  output o = (c, omega); proposed bracket in standardised units c -+ exp(omega).
* Label z = (x_(k) - mu)/sd.  Loss per example:
      (z - c)^2 + rho_tau(|z - c| - exp(omega)),  rho_tau(u) = u (tau - [u < 0]),
  the paper's asymmetric pinball u() (Eq. med_objOS) used as a quantile loss for
  the half-width, tau = 0.99; the batch loss is the mean.
* Adam (Kingma & Ba 2015) with bias correction.
"""
from __future__ import annotations

import math

import numpy as np

SAMPLE = 1024
N_QUANT = 32
N_IN = 36
N_HID = 64
N_OUT = 2
TAU = 0.99

# parameter blocks in storage order: W1 (64x36, row = output unit), b1, W2 (64x64),
# b2, W3 (2x64), b3
SHAPES = [(N_HID, N_IN), (N_HID,), (N_HID, N_HID), (N_HID,), (N_OUT, N_HID), (N_OUT,)]
N_PARAMS = sum(int(np.prod(s)) for s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, off = [], 0
    for s in SHAPES:
        size = int(np.prod(s))
        out.append(theta[off:off + size].reshape(s))
        off += size
    return out


def pack(blocks):
    return np.concatenate([np.asarray(b, dtype=np.float64).ravel() for b in blocks])


def init_params(seed):
    """He-style normal initialisation (std sqrt(2/fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    blocks = []
    for s in SHAPES:
        if len(s) == 2:
            blocks.append(rng.normal(0.0, math.sqrt(2.0 / s[1]), size=s))
        else:
            blocks.append(np.zeros(s))
    return pack(blocks)


def sketch_sample(x):
    """The 1024 strided samples s_j = x[j * floor(n/1024)] (unsorted)."""
    x = np.asarray(x)
    n = x.size
    if n < SAMPLE:
        raise ValueError("the sketch needs n >= 1024")
    stride = n // SAMPLE
    return x[np.arange(SAMPLE) * stride]


def sketch_features(x):
    """(features[36], mu, sd) of the sketch of x, in float64."""
    s = np.sort(sketch_sample(x).astype(np.float64))
    mu = math.fsum(s.tolist()) / SAMPLE
    var = math.fsum(((s - mu) ** 2).tolist()) / SAMPLE
    sd = math.sqrt(var)
    if sd == 0.0:
        sd = 1.0
    q = s[16 + 32 * np.arange(N_QUANT)]
    f = np.empty(N_IN)
    f[:N_QUANT] = (q - mu) / sd
    f[32] = math.asinh((s[0] - mu) / sd)
    f[33] = math.asinh((s[-1] - mu) / sd)
    f[34] = math.asinh(mu / sd)
    f[35] = math.log(sd) / 16.0
    return f, mu, sd


def gelu(u):
    """u * Phi(u), Phi the standard normal CDF."""
    u = np.asarray(u, dtype=np.float64)
    return 0.5 * u * (1.0 + _erf(u / math.sqrt(2.0)))


def gelu_grad(u):
    """d/du [u Phi(u)] = Phi(u) + u phi(u)."""
    u = np.asarray(u, dtype=np.float64)
    Phi = 0.5 * (1.0 + _erf(u / math.sqrt(2.0)))
    phi = np.exp(-0.5 * u * u) / math.sqrt(2.0 * math.pi)
    return Phi + u * phi


_erf = np.vectorize(math.erf, otypes=[np.float64])


def forward(theta, F):
    """Network outputs (B, 2) for features F (B, 36), plus the activations cache."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    F = np.atleast_2d(np.asarray(F, dtype=np.float64))
    u1 = F @ W1.T + b1
    h1 = gelu(u1)
    u2 = h1 @ W2.T + b2
    h2 = gelu(u2)
    o = h2 @ W3.T + b3
    return o, (F, u1, h1, u2, h2)


def loss(o, z, tau=TAU):
    """Mean over the batch of (z-c)^2 + rho_tau(|z-c| - exp(omega))."""
    o = np.atleast_2d(o)
    c, om = o[:, 0], o[:, 1]
    z = np.asarray(z, dtype=np.float64)
    d = z - c
    u = np.abs(d) - np.exp(om)
    rho = u * (tau - (u < 0))
    return float(np.mean(d * d + rho))


def loss_grad_o(o, z, tau=TAU):
    """d loss / d o (B, 2), the derivative of :func:`loss` (subgradient choices:
    sign(0) = 0 and rho' = tau at u = 0)."""
    o = np.atleast_2d(o)
    c, om = o[:, 0], o[:, 1]
    z = np.asarray(z, dtype=np.float64)
    B = o.shape[0]
    d = z - c
    w = np.exp(om)
    u = np.abs(d) - w
    drho = tau - (u < 0)
    g = np.empty_like(o)
    g[:, 0] = (-2.0 * d - drho * np.sign(d)) / B
    g[:, 1] = (-drho * w) / B
    return g


def backward(theta, cache, g_o):
    """Gradient of sum(g_o * o) with respect to the packed parameters."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    F, u1, h1, u2, h2 = cache
    gW3 = g_o.T @ h2
    gb3 = g_o.sum(axis=0)
    g_h2 = g_o @ W3
    g_u2 = g_h2 * gelu_grad(u2)
    gW2 = g_u2.T @ h1
    gb2 = g_u2.sum(axis=0)
    g_h1 = g_u2 @ W2
    g_u1 = g_h1 * gelu_grad(u1)
    gW1 = g_u1.T @ F
    gb1 = g_u1.sum(axis=0)
    return pack([gW1, gb1, gW2, gb2, gW3, gb3])


def loss_and_grad(theta, F, z, tau=TAU):
    o, cache = forward(theta, F)
    return loss(o, z, tau), backward(theta, cache, loss_grad_o(o, z, tau))


def adam_step(theta, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t is the 1-based step); returns (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def propose(theta, x):
    """Proposed bracket (a, b) in the data's units for array x."""
    f, mu, sd = sketch_features(x)
    o, _ = forward(theta, f[None, :])
    c, w = o[0, 0], math.exp(o[0, 1])
    return mu + sd * (c - w), mu + sd * (c + w)
