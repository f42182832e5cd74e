"""Pins of the MLP oracle against finite differences, closed forms and the
bfloat16 definition. CPU only."""

import numpy as np

from oracle import mlp


def test_bf16_rounding_definition():
    # bfloat16 keeps 8 significant bits: 1 + 2^-8 is a tie between 1 and
    # 1 + 2^-7 and goes to the even one (1); 1 + 3*2^-9 rounds up to 1 + 2^-7
    v = mlp.bf16(np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -2.5, 3.4e38]))
    assert v[0] == 1.0 and v[1] == 1.0 and v[2] == 1.0 + 2.0 ** -7
    assert v[3] == -2.5
    assert np.isinf(v[4])          # above the largest finite bfloat16 (3.3895e38)


def test_linear_layer_closed_form():
    rng = np.random.default_rng(0)
    W, b = rng.standard_normal((3, 2)), rng.standard_normal(2)
    x = rng.standard_normal((4, 3))
    y, _ = mlp.forward([(W, b)], x, quantize=False)
    assert np.allclose(y, x @ W + b, rtol=1e-14)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    params = mlp.init_params([5, 7, 7, 3], rng)
    params = [(W, rng.standard_normal(W.shape[1]) * 0.1) for W, _ in params]
    x = rng.standard_normal((6, 5))
    dy = rng.standard_normal((6, 3))
    y, cache = mlp.forward(params, x, quantize=False)
    grads = mlp.backward(params, cache, dy, quantize=False)
    f = lambda ps: float(np.sum(mlp.forward(ps, x, quantize=False)[0] * dy))
    h = 1e-6
    for l in range(3):
        W, b = params[l]
        for idx in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (2, 1)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[idx] += h
            Wm[idx] -= h
            pp = list(params); pp[l] = (Wp, b)
            pm = list(params); pm[l] = (Wm, b)
            fd = (f(pp) - f(pm)) / (2 * h)
            assert abs(fd - grads[l][0][idx]) < 1e-6 * max(1.0, abs(fd))
        bp, bm = b.copy(), b.copy()
        bp[0] += h
        bm[0] -= h
        pp = list(params); pp[l] = (W, bp)
        pm = list(params); pm[l] = (W, bm)
        assert abs((f(pp) - f(pm)) / (2 * h) - grads[l][1][0]) < 1e-6


def test_mse_gradient_and_adam_first_step():
    rng = np.random.default_rng(2)
    y, t = rng.standard_normal((4, 3)), rng.standard_normal((4, 3))
    g = mlp.mse_grad(y, t)
    h = 1e-7
    y2 = y.copy(); y2[1, 2] += h
    assert abs((mlp.mse(y2, t) - mlp.mse(y, t)) / h - g[1, 2]) < 1e-5
    # first Adam step moves every parameter by lr * sign(gradient)
    W = rng.standard_normal((3, 2)); b = rng.standard_normal(2)
    gW = rng.standard_normal((3, 2)); gb = rng.standard_normal(2)
    state = [(np.zeros_like(W), np.zeros_like(W), np.zeros_like(b), np.zeros_like(b))]
    (W1, b1), = mlp.adam([(W, b)], [(gW, gb)], state, 1e-3, 1, eps=0.0)
    assert np.allclose(W1 - W, -1e-3 * np.sign(gW), rtol=1e-12)
    assert np.allclose(b1 - b, -1e-3 * np.sign(gb), rtol=1e-12)
