"""Pins of the bracket-proposal oracle: central finite differences, closed forms of
GELU, and the sketch definition by direct indexing. CPU only."""
import math

import numpy as np
import pytest

from oracle import bracket as ob


def test_param_count():
    assert ob.N_PARAMS == 36 * 64 + 64 + 64 * 64 + 64 + 64 * 2 + 2


def test_gelu_closed_forms():
    assert ob.gelu(0.0) == 0.0
    # Phi(1) = (1 + erf(1/sqrt 2))/2 = 0.8413447460685429...
    assert ob.gelu(1.0) == pytest.approx(0.8413447460685429, rel=1e-15)
    assert ob.gelu(-1.0) == pytest.approx(-(1 - 0.8413447460685429), rel=1e-14)
    assert ob.gelu_grad(0.0) == 0.5
    for u in (-3.0, -0.7, 0.2, 2.5):
        h = 1e-6
        fd = (ob.gelu(u + h) - ob.gelu(u - h)) / (2 * h)
        assert ob.gelu_grad(u) == pytest.approx(fd, rel=1e-8)


def test_backward_matches_central_differences():
    rng = np.random.default_rng(21)
    theta = ob.init_params(3) + rng.normal(0, 0.05, ob.N_PARAMS)
    F = rng.normal(size=(5, ob.N_IN))
    z = rng.normal(size=5)
    _, g = ob.loss_and_grad(theta, F, z)
    idx = rng.choice(ob.N_PARAMS, 60, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (ob.loss(ob.forward(tp, F)[0], z) - ob.loss(ob.forward(tm, F)[0], z)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_loss_closed_form():
    # c = 0, omega = 0 (w = 1): z = 3 -> d = 3, u = 2 > 0 -> 9 + 0.99*2
    o = np.array([[0.0, 0.0]])
    assert ob.loss(o, [3.0]) == pytest.approx(9 + 0.99 * 2)
    # z = 0.5 -> u = -0.5 -> 0.25 + (0.99 - 1)(-0.5)
    assert ob.loss(o, [0.5]) == pytest.approx(0.25 + 0.005)


def test_adam_first_step_is_lr_times_sign():
    """After bias correction the first Adam step is lr * g / (|g| + eps)."""
    th = np.zeros(4)
    g = np.array([1.0, -2.0, 0.5, 0.0])
    th1, m, v = ob.adam_step(th, g, np.zeros(4), np.zeros(4), 1, lr=1e-3)
    assert th1 == pytest.approx(-1e-3 * g / (np.abs(g) + 1e-8))


def test_sketch_indexing_and_features():
    n = 1024 * 7 + 5
    x = np.arange(n, dtype=np.float32)[::-1].copy()
    s = ob.sketch_sample(x)
    assert s.size == 1024
    assert s[0] == x[0] and s[1] == x[7] and s[1023] == x[1023 * 7]
    f, mu, sd = ob.sketch_features(x)
    srt = np.sort(s.astype(np.float64))
    assert mu == pytest.approx(srt.mean())
    assert sd == pytest.approx(srt.std())
    assert f[0] == pytest.approx((srt[16] - mu) / sd)
    assert f[31] == pytest.approx((srt[16 + 32 * 31] - mu) / sd)
    assert f[32] == pytest.approx(math.asinh((srt[0] - mu) / sd))
    assert f[35] == pytest.approx(math.log(sd) / 16)


def test_constant_array_features_finite():
    f, mu, sd = ob.sketch_features(np.full(4096, 2.5, dtype=np.float32))
    assert sd == 1.0 and np.all(np.isfinite(f))


def test_philox_known_answer_vectors():
    """Philox4x32-10 against the published known-answer vectors (Random123, Salmon et al.)."""
    import json
    import os
    from oracle.philox import philox4x32_10
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.json")))
    for v in g["vectors"]:
        out = philox4x32_10([int(c, 16) for c in v["counter"]], [int(k, 16) for k in v["key"]])
        assert ["%08x" % o for o in out] == v["output"]
