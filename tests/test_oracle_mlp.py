"""Pins of the MLP oracle: bfloat16 rounding against torch's conversion, SiLU'
against a central difference, back-propagated gradients against central
differences of the loss, and AdamW against its closed form."""
import numpy as np
import pytest

from oracle import mlp


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10 ** rng.uniform(-6, 6, 20000),
                        [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -1.0 - 2 ** -8, 0.0, 65504.0]])
    x32 = x.astype(np.float32)
    ref = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x32), ref)
    # ties to even: 1 + 2^-8 is half-way between 1 and 1 + 2^-7
    assert mlp.bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert mlp.bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6


def test_dsilu_is_derivative():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.allclose(mlp.dsilu(z), fd, rtol=1e-8, atol=1e-9)
    assert mlp.silu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.silu(np.array([30.0]))[0] - 30.0) < 1e-10


def _net(rng, dims):
    return [(rng.standard_normal((o, i)) / np.sqrt(i), 0.1 * rng.standard_normal(o))
            for o, i in dims]


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    dims = [(16, 5), (16, 16), (4, 16)]
    layers = _net(rng, dims)
    X = rng.standard_normal((7, 5))
    T = rng.standard_normal((7, 4))
    loss, grads, _ = mlp.loss_and_grads(layers, X, T, n_valid=3, m_valid=6, bf=False)
    h = 1e-6
    for l, (W, b) in enumerate(layers):
        for idx in [(0, 0), (3, 2), (W.shape[0] - 1, W.shape[1] - 1)]:
            Wp = [(w.copy(), bb.copy()) for w, bb in layers]
            Wm = [(w.copy(), bb.copy()) for w, bb in layers]
            Wp[l][0][idx] += h
            Wm[l][0][idx] -= h
            lp = mlp.loss_and_grads(Wp, X, T, 3, 6, bf=False)[0]
            lm = mlp.loss_and_grads(Wm, X, T, 3, 6, bf=False)[0]
            assert grads[l][0][idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)
        for k in (0, len(b) - 1):
            Wp = [(w.copy(), bb.copy()) for w, bb in layers]
            Wm = [(w.copy(), bb.copy()) for w, bb in layers]
            Wp[l][1][k] += h
            Wm[l][1][k] -= h
            lp = mlp.loss_and_grads(Wp, X, T, 3, 6, bf=False)[0]
            lm = mlp.loss_and_grads(Wm, X, T, 3, 6, bf=False)[0]
            assert grads[l][1][k] == pytest.approx((lp - lm) / (2 * h), rel=1e-5, abs=1e-9)
    # masked outputs and rows carry no gradient into the output bias
    assert np.all(grads[-1][1][3:] == 0)


def test_adamw_closed_form():
    w = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -0.1, 0.0])
    m = np.zeros(3)
    v = np.zeros(3)
    w1, m1, v1 = mlp.adamw(w, g, m, v, t=1, lr=0.01, wd=0.1, eps=1e-8)
    # first step: m_hat = g, v_hat = g^2 -> update lr (g/(|g| + eps) + wd w)
    expect = w - 0.01 * (g / (np.abs(g) + 1e-8) + 0.1 * w)
    assert np.allclose(w1, expect, rtol=1e-12)
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)
    # zero gradient: pure decoupled decay w (1 - lr wd)
    assert w1[2] == pytest.approx(0.5 * (1 - 0.01 * 0.1), rel=1e-12)


def test_flatten_roundtrip():
    rng = np.random.default_rng(2)
    dims = [(16, 16), (16, 16), (16, 16)]
    parts = _net(rng, dims)
    back = mlp.unflatten(mlp.flatten(parts), dims)
    for (W, b), (W2, b2) in zip(parts, back):
        assert np.array_equal(W, W2) and np.array_equal(b, b2)
