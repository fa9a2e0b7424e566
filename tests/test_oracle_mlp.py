"""Pins of the learned-residual oracle (oracle/mlp.py) against facts outside
its own code: exact rational cell arithmetic, a network whose output has a
closed form, central finite differences of the loss, Adam's closed-form first
steps, and bfloat16 rounding of hand-checked values."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import mlp


def _coded_planes(W, H):
    """C and grads whose every value encodes (quantity, channel, x, y)."""
    ys, xs = np.mgrid[0:H, 0:W]
    code = lambda q, c: ((q * 3 + c) * 1000.0 + ys) * 1000.0 + xs
    C = np.stack([code(0, c) for c in range(3)])
    G = np.stack([np.stack([code(d + 1, c) for c in range(3)]) for d in range(3)])
    return C, G


def _cell_exact(X, W, W2):
    """floor of x = (2X + 1) W / (2 W2) - 1/2 in exact rationals, clamped, and t."""
    x = Fraction((2 * X + 1) * W - W2, 2 * W2)
    i = min(max(x.numerator // x.denominator, 0), W - 2)
    return i, x - i


@pytest.mark.parametrize("W,H,W2,H2", [(9, 7, 36, 28), (16, 12, 24, 18), (5, 4, 37, 11), (2, 2, 3, 5),
                                       (30, 17, 30, 17)])
def test_features_decode(ora, W, H, W2, H2):
    C, G = _coded_planes(W, H)
    rng = np.random.default_rng(W2 * H2)
    pix = np.stack([rng.integers(0, W2, 60), rng.integers(0, H2, 60)], 1)
    pix[:4] = [[0, 0], [W2 - 1, 0], [0, H2 - 1], [W2 - 1, H2 - 1]]
    f = mlp.features(C, G, W2, H2, pix)
    assert f.shape == (len(pix), 50)
    for m, (X, Y) in enumerate(pix):
        i, t = _cell_exact(int(X), W, W2)
        j, u = _cell_exact(int(Y), H, H2)
        for k, (di, dj) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
            for q in range(4):
                for c in range(3):
                    v = int(f[m, 12 * k + 3 * q + c])
                    assert v == ((q * 3 + c) * 1000 + j + dj) * 1000 + i + di
        assert abs(f[m, 48] - float(t)) < 1e-12 and abs(f[m, 49] - float(u)) < 1e-12
    full = mlp.features(C, G, W2, H2)
    Y, X = np.divmod(np.arange(W2 * H2), W2)
    assert np.array_equal(full[Y * W2 + X][:10], mlp.features(C, G, W2, H2, np.stack([X, Y], 1))[:10])


def test_zero_last_layer_is_the_spline(ora):
    rng = np.random.default_rng(0)
    C = rng.uniform(0, 1, (3, 11, 13))
    G = rng.normal(0, 0.3, (3, 3, 11, 13))
    p = mlp.unpack(rng.normal(0, 0.2, mlp.N_PARAMS).copy())
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    theta = mlp.pack(p)
    assert np.array_equal(mlp.upscale(C, G, 26, 22, theta), ora.upscale(C, G, 26, 22))


def test_relu_network_closed_form():
    """W1 copies feature k (k < 50) into unit k with offset b1[k]; units 50..63
    read -t; W2 = I; W3 sums the units with weights (1, 2, -1).  Then
    r_c = w_c sum_k relu(z1_k) + b3_c, since relu(relu(z)) = relu(z)."""
    p = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    rng = np.random.default_rng(1)
    for k in range(50):
        p["W1"][k, k] = 1.0
    p["W1"][50:, 48] = -1.0
    p["b1"][:] = rng.normal(0, 0.5, 64)
    p["W2"][:] = np.eye(64)
    w = (1.0, 2.0, -1.0)
    for c in range(3):
        p["W3"][c, :] = w[c]
    p["b3"][:] = (0.1, -0.2, 0.3)
    f = rng.normal(0, 1, (7, 50))
    r, _ = mlp.forward(mlp.pack(p), f)
    for m in range(7):
        s = 0.0
        for k in range(64):
            z = (f[m, k] if k < 50 else -f[m, 48]) + p["b1"][k]
            s += z if z > 0 else 0.0
        for c in range(3):
            assert abs(r[m, c] - (w[c] * s + p["b3"][c])) < 1e-12


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    M = 12
    f = rng.normal(0, 1, (M, 50))
    base = rng.uniform(0, 1, (M, 3))
    target = rng.uniform(0, 1, (M, 3))
    for _ in range(20):
        theta = rng.normal(0, 0.3, mlp.N_PARAMS)
        _, s = mlp.forward(theta, f)
        if min(np.abs(s["z1"]).min(), np.abs(s["z2"]).min()) > 1e-4:
            break
    g, L = mlp.gradient(theta, f, base, target)
    assert abs(L - mlp.loss(theta, f, base, target)) < 1e-15
    eps = 1e-6
    fd = np.empty_like(theta)
    for k in range(mlp.N_PARAMS):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += eps
        tm[k] -= eps
        fd[k] = (mlp.loss(tp, f, base, target) - mlp.loss(tm, f, base, target)) / (2 * eps)
    assert np.abs(g - fd).max() <= 1e-7 * (1.0 + np.abs(fd).max())
    # every block of the gradient is exercised
    for name, a in mlp.unpack(g).items():
        assert np.abs(a).max() > 0, name


def test_adam_closed_form_first_steps():
    """With bias correction, a constant gradient g gives m_hat = g and
    v_hat = g^2 at every step, so each update is -lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    g = rng.normal(0, 1, 100)
    theta = rng.normal(0, 1, 100)
    m = np.zeros(100)
    v = np.zeros(100)
    lr, eps = 1e-3, 1e-8
    t = theta
    for step in (1, 2, 3):
        t_new, m, v = mlp.adam(t, m, v, g, step, lr, eps=eps)
        np.testing.assert_allclose(t_new - t, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-18)
        t = t_new
    # first moment after two steps: (1 - beta1^2) g
    _, m2, v2 = mlp.adam(theta, *mlp.adam(theta, np.zeros(100), np.zeros(100), g, 1, lr)[1:], g, 2, lr)
    np.testing.assert_allclose(m2, (1 - 0.9 ** 2) * g, rtol=1e-14)
    np.testing.assert_allclose(v2, (1 - 0.999 ** 2) * g * g, rtol=1e-12)


def test_bf16_round():
    u = 2.0 ** -8
    cases = {1.0: 1.0, 1.0 + u: 1.0,                        # tie -> even (down)
             1.0 + 3 * u: 1.0 + 4 * u,                       # tie -> even (up)
             1.0 + u + 2.0 ** -20: 1.0 + 2 * u,              # above the tie
             -(1.0 + 3 * u): -(1.0 + 4 * u), 0.0: 0.0, 3.0: 3.0, 1.0 / 3.0: 0.333984375,
             65504.0: 65536.0}
    for a, want in cases.items():
        assert mlp.bf16_round(np.array([a]))[0] == want, a
    x = np.random.default_rng(4).normal(0, 10, 10000)
    r = mlp.bf16_round(x)
    assert np.all(np.abs(r - x) <= u * np.abs(x) * (1 + 1e-6))
    assert np.array_equal(mlp.bf16_round(r), r)
    # 8 significant bits: r * 2^(7 - exponent) is an integer
    e = np.floor(np.log2(np.abs(r[r != 0])))
    assert np.all(np.mod(r[r != 0] * 2.0 ** (7 - e), 1.0) == 0)
