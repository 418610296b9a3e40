"""The per-element gradient tolerance of the GPU parity tests (tests/gradbound.py) is
checked on the CPU from both sides: a float32 evaluation of the network's gradient
(numpy, another summation order than the GPU's) lies inside it on every element, and
plausible mistakes planted in a copy of the float64 gradient fall outside it."""
import math

import numpy as np

import gradbound
from oracle import bracket as ob


def float32_gradient(theta, F, z, tau=ob.TAU):
    """The loss gradient formed entirely in float32 (GELU and its slope evaluated in
    float64 and rounded, as a float32 library call would be to within an ulp or two)."""
    f32 = np.float32
    W1, b1, W2, b2, W3, b3 = (b.astype(f32) for b in ob.unpack(theta))
    F = F.astype(f32)
    z = z.astype(f32)
    B = F.shape[0]

    def gelu(u):
        return ob.gelu(u.astype(np.float64)).astype(f32)

    def gelu_grad(u):
        return ob.gelu_grad(u.astype(np.float64)).astype(f32)

    u1 = F @ W1.T + b1
    h1 = gelu(u1)
    u2 = h1 @ W2.T + b2
    h2 = gelu(u2)
    o = h2 @ W3.T + b3
    c, om = o[:, 0], o[:, 1]
    d = z - c
    w = np.exp(om)
    uu = np.abs(d) - w
    drho = (f32(tau) - (uu < 0)).astype(f32)
    g_o = np.empty_like(o)
    g_o[:, 0] = (f32(-2.0) * d - drho * np.sign(d)) / f32(B)
    g_o[:, 1] = (-drho * w) / f32(B)
    g_h2 = g_o @ W3
    g_u2 = g_h2 * gelu_grad(u2)
    g_h1 = g_u2 @ W2
    g_u1 = g_h1 * gelu_grad(u1)
    blocks = [g_u1.T @ F, g_u1.sum(axis=0), g_u2.T @ h1, g_u2.sum(axis=0), g_o.T @ h2, g_o.sum(axis=0)]
    return np.concatenate([b.astype(np.float64).ravel() for b in blocks])


def problem(seed, B):
    rng = np.random.default_rng(seed)
    theta = ob.init_params(seed) + rng.normal(0, 0.05, ob.N_PARAMS)
    theta = theta.astype(np.float32).astype(np.float64)
    F = rng.normal(size=(B, ob.N_IN)).astype(np.float32).astype(np.float64)
    z = gradbound.kink_free_labels(theta, F, rng, rng.normal(size=B)).astype(np.float64)
    return theta, F, z


def test_float32_gradient_lies_inside_the_bound():
    for seed, B in ((31, 777), (32, 64), (33, 512)):
        theta, F, z = problem(seed, B)
        _, g64 = ob.loss_and_grad(theta, F, z)
        g32 = float32_gradient(theta, F, z)
        tol = gradbound.gradient_bound(theta, F, z) + 1e-4 * np.abs(g64)
        assert np.all(np.abs(g32 - g64) <= tol)
        # the bound is not vacuous: it stays far below the gradient's own size
        assert np.median(tol / (np.abs(g64) + 1e-30)) < 0.02


def test_planted_gradient_mistakes_fall_outside_the_bound():
    theta, F, z = problem(34, 777)
    o, cache = ob.forward(theta, F)
    g64 = ob.backward(theta, cache, ob.loss_grad_o(o, z))
    tol = gradbound.gradient_bound(theta, F, z) + 1e-4 * np.abs(g64)
    shapes = ob.SHAPES
    offs = np.cumsum([0] + [int(np.prod(s)) for s in shapes])

    def caught(g):
        return np.any(np.abs(g - g64) > tol)

    # 1. two rows of W1's gradient exchanged (a mis-indexed output unit)
    g = g64.copy()
    gW1 = g[offs[0]:offs[1]].reshape(shapes[0])
    gW1[[3, 17]] = gW1[[17, 3]]
    assert caught(g)
    # 2. one column of W2's gradient taken from its neighbour (a mis-indexed input)
    g = g64.copy()
    gW2 = g[offs[2]:offs[3]].reshape(shapes[2])
    gW2[:, 5] = gW2[:, 6]
    assert caught(g)
    # 3. the u*phi(u) term of GELU' dropped for one first-layer unit
    F_, u1, h1, u2, h2 = cache
    W1, b1, W2, b2, W3, b3 = ob.unpack(theta)
    g_o = ob.loss_grad_o(o, z)
    g_u2 = (g_o @ W3) * ob.gelu_grad(u2)
    g_h1 = g_u2 @ W2
    slope = ob.gelu_grad(u1)
    Phi = 0.5 * (1.0 + np.vectorize(math.erf)(u1[:, 9] / math.sqrt(2.0)))
    slope[:, 9] = Phi
    g_u1 = g_h1 * slope
    g = g64.copy()
    g[offs[0]:offs[1]] = (g_u1.T @ F_).ravel()
    g[offs[1]:offs[2]] = g_u1.sum(axis=0)
    assert caught(g)
    # 4. the output bias's gradient with one row's contribution counted twice
    g = g64.copy()
    b = int(np.argmax(np.abs(g_o[:, 0])))
    g[offs[5]] += g_o[b, 0]
    assert caught(g)


def test_adam_bound_holds_for_a_float32_update():
    theta, F, z = problem(35, 512)
    _, g64 = ob.loss_and_grad(theta, F, z)
    g32 = float32_gradient(theta, F, z).astype(np.float32)
    lr = np.float32(1e-3)
    w0 = theta.astype(np.float32)
    m = np.float32(0.1) * g32
    v = np.float32(0.001) * g32 * g32
    c1, c2 = np.float32(1 - 0.9), np.float32(1 - 0.999)
    w1 = w0 - lr * (m / c1) / (np.sqrt(v / c2) + np.float32(1e-8))
    w1_64, _, _ = ob.adam_step(theta, g64, np.zeros_like(g64), np.zeros_like(g64), 1, lr=1e-3)
    gb = gradbound.gradient_bound(theta, F, z) + 1e-4 * np.abs(g64)
    tol = gradbound.adam_first_step_bound(g64, gb, w1_64, 1e-3)
    assert np.all(np.abs(w1.astype(np.float64) - w1_64) <= tol)
    # a step taken with the sign of one resolved gradient element flipped is caught
    j = int(np.argmax(np.abs(g64) / gb))
    w_bad = w1.astype(np.float64).copy()
    w_bad[j] = theta[j] + 1e-3 * np.sign(g64[j])
    assert np.abs(w_bad[j] - w1_64[j]) > tol[j]
