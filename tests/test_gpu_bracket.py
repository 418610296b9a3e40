"""GPU parity of the learned-bracket pieces: Philox generator, sketch features, network
forward / gradient / Adam against the float64 oracle, and selections that use a
proposed bracket (results must not depend on the proposal)."""
import os

import numpy as np
import pytest
import torch

import synth
from oracle import bracket as ob
from oracle import philox as oph
from oracle import select as osel

pytestmark = pytest.mark.gpu

MODEL = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1104_2732_gb300",
                     "bracket_model.bin")


@pytest.fixture(scope="module")
def ctx(lib):
    c = lib.Context()
    yield c
    c.close()


def bits(v):
    return np.asarray(v, dtype=np.float32).view(np.uint32)


def test_philox_matches_oracle_and_known_answers(ctx):
    rng = np.random.default_rng(100)
    m = 300
    ctr = rng.integers(0, 2 ** 32, (m, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, (m, 2), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    key[0] = 0
    ctr[1] = 0xFFFFFFFF
    key[1] = 0xFFFFFFFF
    got = ctx.philox(torch.from_numpy(ctr.view(np.int32)).cuda(), torch.from_numpy(key.view(np.int32)).cuda())
    got = got.cpu().numpy().view(np.uint32).reshape(m, 4)
    for i in range(m):
        assert list(got[i]) == oph.philox4x32_10(ctr[i], key[i])
    assert ["%08x" % v for v in got[0]] == ["6627e8d5", "e169c58d", "bc57ac4c", "9b00dbd8"]


def test_generator_deterministic_and_distributed(ctx):
    x = torch.empty(1 << 20, device="cuda")
    y = torch.empty(1 << 20, device="cuda")
    ctx.generate_training_array(x, 0, seed=7)
    ctx.generate_training_array(y, 0, seed=7)
    assert torch.equal(x, y)
    ctx.generate_training_array(y, 0, seed=8)
    assert not torch.equal(x, y)
    v = x.double()
    assert abs(v.mean().item()) < 0.01 and abs(v.std().item() - 1) < 0.01
    ctx.generate_training_array(y, 2, p0=0.5, seed=9)                   # lognormal(0, 0.5)
    assert abs(torch.log(y.double()).std().item() - 0.5) < 0.01
    ctx.generate_training_array(y, 3, p0=0.25, p1=10.0, p2=1.0, seed=10)  # 25% at N(10, 1)
    assert abs((y > 5).double().mean().item() - 0.25) < 0.01
    ctx.generate_training_array(y, 1, p0=3.0, seed=11)                   # Student-t, nu = 3
    q = torch.quantile(y[:100000].double(), torch.tensor([0.975], dtype=torch.float64, device="cuda")).item()
    assert abs(q - 3.182) < 0.1


def test_features_match_oracle(ctx):
    for seed, n in ((200, 5000), (201, 1 << 20), (202, 123457)):
        x = synth.training_array(seed, n=n)
        f, musd = ctx.bracket_features(torch.from_numpy(x).cuda())
        f64, mu, sd = ob.sketch_features(x)
        assert musd.cpu().numpy() == pytest.approx([mu, sd], rel=1e-12)
        assert np.allclose(f.cpu().numpy(), f64, rtol=1e-6, atol=1e-6)


def random_weights(seed):
    return (ob.init_params(seed) + np.random.default_rng(seed).normal(0, 0.05, ob.N_PARAMS)).astype(np.float32)


def test_forward_and_gradient_match_float64(ctx):
    """Forward outputs within 1e-4, the loss within 1e-4 relative, and every one of the
    6658 gradient elements g_j within (B u + 1e-4) sum_b |c_bj| + 1e-4 |g_j| of the float64
    oracle's, c_bj the per-row contributions and B = 777 rows (tests/gradbound.py derives
    it: the batch sum's rounding plus a per-row chain budget).  Labels sit at least 0.05
    from the loss's kinks, so float32 and float64 take the same subgradient branch."""
    import gradbound
    rng = np.random.default_rng(203)
    w = random_weights(5)
    ctx.set_bracket_model(w)
    B = 777
    F = rng.normal(size=(B, 36)).astype(np.float32)
    w64, F64 = w.astype(np.float64), F.astype(np.float64)
    Z = gradbound.kink_free_labels(w64, F64, rng, rng.normal(size=B))
    Ft, Zt = torch.from_numpy(F).cuda(), torch.from_numpy(Z).cuda()
    out = ctx.bracket_forward(Ft).cpu().numpy()
    o64, _ = ob.forward(w64, F64)
    assert np.allclose(out, o64, rtol=1e-4, atol=1e-4)
    g, loss = ctx.bracket_grad(Ft, Zt)
    l64, g64 = ob.loss_and_grad(w64, F64, Z.astype(np.float64))
    assert loss.item() == pytest.approx(l64, rel=1e-4)
    g = g.cpu().numpy().astype(np.float64)
    tol = gradbound.gradient_bound(w64, F64, Z.astype(np.float64)) + 1e-4 * np.abs(g64)
    err = np.abs(g - g64)
    worst = int(np.argmax(err / tol))
    assert np.all(err <= tol), (worst, g[worst], g64[worst], tol[worst])


def test_training_reduces_loss_and_adam_step(ctx):
    """The first Adam step from zero moments equals the oracle's on every parameter,
    within the bound that the float32 gradient's own bound implies for the update
    lr * g / (|g| + eps) (tests/gradbound.py); then many steps reduce the loss."""
    import gradbound
    rng = np.random.default_rng(204)
    w = random_weights(6)
    B = 512
    F = rng.normal(size=(B, 36)).astype(np.float32)
    w64, F64 = w.astype(np.float64), F.astype(np.float64)
    Z = gradbound.kink_free_labels(w64, F64, rng, 0.3 * F64[:, 0] - 0.2 * F64[:, 5] + 0.1 * rng.normal(size=B))
    Ft, Zt = torch.from_numpy(F).cuda(), torch.from_numpy(Z).cuda()
    ctx.set_bracket_model(w)
    ctx.bracket_train(Ft, Zt, batch=B, steps=1, lr=1e-3, seed=0)
    w1 = ctx.get_bracket_model().astype(np.float64)
    Z64 = Z.astype(np.float64)
    _, g64 = ob.loss_and_grad(w64, F64, Z64)
    w1_64, _, _ = ob.adam_step(w64, g64, np.zeros_like(g64), np.zeros_like(g64), 1, lr=1e-3)
    gb = gradbound.gradient_bound(w64, F64, Z64) + 1e-4 * np.abs(g64)
    tol = gradbound.adam_first_step_bound(g64, gb, w1_64, 1e-3)
    err = np.abs(w1 - w1_64)
    worst = int(np.argmax(err / tol))
    assert np.all(err <= tol), (worst, w1[worst], w1_64[worst], g64[worst], tol[worst])
    # many steps: the loss falls
    ctx.set_bracket_model(w)
    hist = ctx.bracket_train(Ft, Zt, batch=128, steps=400, lr=3e-3, seed=1)
    assert np.mean(hist[-20:]) < 0.5 * np.mean(hist[:20])


def constant_model(c, omega):
    """A network whose output is (c, omega) whatever the features."""
    w = np.zeros(ob.N_PARAMS, np.float32)
    w[-2] = c
    w[-1] = omega
    return w


@pytest.mark.parametrize("c,omega,expect", [
    (0.0, np.log(0.05), None),     # tight around the sample mean
    (0.0, np.log(3.0), 1),         # wide: valid, Kelley from the proposal
    (50.0, 0.0, 2),                # far above: a fails, (m, b]
    (-50.0, 0.0, 2),               # far below: b fails, (a, M]
    (0.0, np.log(1e-6), None),     # almost empty bracket
    (0.0, 25.0, 1),                # covers everything
])
def test_select_with_proposed_bracket_is_exact(ctx, c, omega, expect):
    ctx.set_bracket_model(constant_model(c, omega))
    ctx.set_config(use_learned=1)
    try:
        for fam in synth.HEAVY_FAMILIES:
            x = synth.heavy_mixture(fam, 300001, seed=205)
            xt = torch.from_numpy(x).cuda()
            k = (x.size + 1) // 2
            r = ctx.select_kth(xt, k).cpu().numpy()[0]
            st = ctx.last_stats()
            assert bits(r) == bits(osel.select_kth(x, k)), (fam, c, omega, st)
            assert st["learned"] in (1, 2)
            if expect is not None:
                assert st["learned"] == expect
        # a non-median rank ignores the model
        x = synth.paper_distribution("normal", 300001, seed=206)
        r = ctx.select_kth(torch.from_numpy(x).cuda(), 1000).cpu().numpy()[0]
        assert bits(r) == bits(osel.select_kth(x, 1000)) and ctx.last_stats()["learned"] == 0
    finally:
        ctx.set_config(use_learned=0)


def test_proposal_matches_oracle_network(ctx):
    w = random_weights(7)
    ctx.set_bracket_model(w)
    x = synth.training_array(207, n=1 << 18)
    p = ctx.bracket_propose(torch.from_numpy(x).cuda()).cpu().numpy()
    a, b = ob.propose(w.astype(np.float64), x)
    assert p[2] == 1.0
    assert p[0] == pytest.approx(a, rel=1e-4, abs=1e-4 * abs(b - a))
    assert p[1] == pytest.approx(b, rel=1e-4, abs=1e-4 * abs(b - a))


def test_model_checkpoint_roundtrip(ctx, tmp_path):
    w = random_weights(8)
    ctx.set_bracket_model(w)
    path = str(tmp_path / "m.bin")
    ctx.save_bracket_model(path)
    ctx.set_bracket_model(np.zeros_like(w))
    ctx.load_bracket_model(path)
    assert np.array_equal(ctx.get_bracket_model(), w)
    with open(path, "r+b") as f:
        f.write(b"XXXXXXXX")
    with pytest.raises(Exception):
        ctx.load_bracket_model(path)


def test_checkpoint_keeps_optimizer_state_for_resume(ctx, lib, tmp_path):
    """A checkpoint holds the Adam step and both moments besides the weights: after two
    training steps the file records step 2 and non-zero moments, and a fresh context that
    loads it writes the same bytes back, so training resumes from step 2."""
    from paper_1104_2732_gb300 import train_bracket as tb
    rng = np.random.default_rng(209)
    B = 256
    F = rng.normal(size=(B, 36)).astype(np.float32)
    Z = (0.3 * F[:, 0] + 0.1 * rng.normal(size=B)).astype(np.float32)
    ctx.set_bracket_model(random_weights(9))
    ctx.bracket_train(torch.from_numpy(F).cuda(), torch.from_numpy(Z).cuda(), batch=B, steps=2, lr=1e-3, seed=0)
    p1, p2 = str(tmp_path / "a.bin"), str(tmp_path / "b.bin")
    ctx.save_bracket_model(p1)
    raw = open(p1, "rb").read()
    n = ob.N_PARAMS
    assert len(raw) == 8 + 20 + 8 + 12 * n
    assert tb.checkpoint_step(p1) == 2
    body = np.frombuffer(raw[36:], dtype="<f4").reshape(3, n)
    assert np.array_equal(body[0], ctx.get_bracket_model())
    assert np.count_nonzero(body[1]) > n // 2 and np.count_nonzero(body[2]) > n // 2
    c2 = lib.Context()
    try:
        c2.load_bracket_model(p1)
        c2.save_bracket_model(p2)
    finally:
        c2.close()
    assert open(p2, "rb").read() == raw


@pytest.mark.skipif(not os.path.exists(MODEL), reason="no trained model in the package")
def test_trained_model_saves_passes_on_held_out_arrays(ctx):
    """Held-out arrays (generator seeds 2e6 + i): the learned start's median equals the
    plain start's and the oracle's bit for bit, with fewer passes on average than from the
    data's extremes."""
    from paper_1104_2732_gb300 import train_bracket as tb
    ctx.load_bracket_model(MODEL)
    rng = np.random.default_rng(2 * 10 ** 6)
    buf = torch.empty(1 << 24, device="cuda")
    plain, learned = [], []
    for i in range(60):
        n, fam, p0, p1, p2, loc, scale = tb.draw_params(rng)
        x = buf[:n]
        ctx.generate_training_array(x, fam, p0, p1, p2, loc, scale, seed=2 * 10 ** 6 + i)
        k = (n + 1) // 2
        ctx.set_config(use_learned=0)
        r0 = ctx.select_kth(x, k).clone()
        plain.append(ctx.last_stats()["passes"])
        ctx.set_config(use_learned=1)
        r1 = ctx.select_kth(x, k).clone()
        learned.append(ctx.last_stats()["passes"])
        assert torch.equal(r0.view(torch.int32), r1.view(torch.int32))
        xh = x.cpu().numpy()
        assert bits(r1.cpu().numpy()[0]) == bits(osel.select_kth(xh, k)), (i, n, fam)
    ctx.set_config(use_learned=0)
    assert np.mean(learned) < np.mean(plain)
