"""The comparison rules of helpers_mlp hold for an emulation of the kernels'
precision in numpy (BF16 narrowing where the kernels narrow: features, h1, h2,
d2, d1; FP32 sums in
another order), and they are tight enough to catch plausible kernel mistakes
(a dropped bias, a transposed W2, a feature slot off by one)."""
import numpy as np

from helpers_mlp import bf16_params, forward_reference, gradient_reference, q, random_theta
from oracle import mlp


def _emulate(theta, f, base=None, target=None, transpose_w2=False, drop_b2=False, shift=0):
    p = {k: np.asarray(v, np.float32) for k, v in mlp.unpack(theta).items()}
    bf = lambda a: q(np.asarray(a, np.float32)).astype(np.float32)
    fb = bf(f)
    if shift:
        fb = np.roll(fb, shift, axis=1)
    z1 = (fb @ bf(p["W1"]).T).astype(np.float32) + p["b1"]
    h1 = bf(np.maximum(z1, 0))
    z2 = (h1 @ bf(p["W2"]).T).astype(np.float32) + (0 if drop_b2 else p["b2"])
    h2 = bf(np.maximum(z2, 0))
    r = (h2 @ bf(p["W3"]).T).astype(np.float32) + p["b3"]
    out = dict(r=r, z1=z1, z2=z2)
    if base is not None:
        M = f.shape[0]
        e = (np.float32(base) + r - np.float32(target)).astype(np.float32)
        d3 = e * np.float32(2.0 / (3 * M))
        d2b = bf((d3 @ bf(p["W3"])) * (z2 > 0))
        W2 = bf(p["W2"]).T if transpose_w2 else bf(p["W2"])
        d1b = bf((d2b @ W2) * (z1 > 0))
        g = {"W3": d3.T @ h2, "b3": d3.sum(0), "W2": d2b.T @ h1, "b2": d2b.sum(0), "W1": d1b.T @ fb,
             "b1": d1b.sum(0)}
        out["g"] = mlp.pack(g)
        out["L"] = float(np.sum(e.astype(np.float64) ** 2) / e.size)
    return out


def _data(seed, M=4000):
    rng = np.random.default_rng(seed)
    f = np.concatenate([rng.normal(0, 1.0, (M, 48)), rng.uniform(-0.4, 1.4, (M, 2))], 1)
    theta = bf16_params(random_theta(rng))
    base = rng.uniform(0, 1, (M, 3))
    target = base + rng.normal(0, 0.05, (M, 3))
    return theta, f, base, target


def test_forward_rule_holds_and_is_tight():
    theta, f, _, _ = _data(0)
    ref = forward_reference(theta, f)
    k = (ref["keep"])
    assert k.mean() > 0.95
    emu = _emulate(theta, f)
    err = np.abs(emu["r"] - ref["r"])[k]
    assert np.all(err <= ref["e3"][k])
    # the bound is small against the residual (median below 0.5 %)
    assert np.median(ref["e3"][k] / (np.abs(ref["r"][k]) + 1e-2)) < 5e-3
    for bad in (dict(drop_b2=True), dict(shift=1)):
        wrong = _emulate(theta, f, **bad)
        assert np.mean(np.abs(wrong["r"] - ref["r"])[k] > ref["e3"][k]) > 0.5, bad


def test_gradient_rule_holds_and_is_tight():
    theta, f, base, target = _data(1)
    f = q(f)
    keep = forward_reference(theta, f)["keep"]
    f, base, target = f[keep], base[keep], target[keep]
    g, bound, L, eL = gradient_reference(theta, f, base, target)
    emu = _emulate(theta, f, base, target)
    assert np.all(np.abs(emu["g"] - g) <= bound)
    assert abs(emu["L"] - L) <= eL
    rel = np.median(bound / (np.abs(g) + 1e-12))
    assert rel < 0.05, rel
    wrong = _emulate(theta, f, base, target, transpose_w2=True)
    gw = mlp.unpack(wrong["g"])["W1"]
    assert np.mean(np.abs(gw - mlp.unpack(g)["W1"]) > mlp.unpack(bound)["W1"]) > 0.5


def test_quantized_oracle_is_exact_on_representable_values():
    """With dyadic weights and inputs of few bits every intermediate is a BF16
    value, so quantising changes nothing."""
    rng = np.random.default_rng(2)
    p = {"W1": rng.integers(-2, 3, (64, 50)) / 8.0, "b1": rng.integers(-2, 3, 64) / 8.0,
         "W2": rng.integers(-1, 2, (64, 64)) / 16.0, "b2": np.zeros(64),
         "W3": rng.integers(-1, 2, (3, 64)) / 4.0, "b3": np.zeros(3)}
    theta = mlp.pack(p)
    f = rng.integers(-2, 3, (5, 50)) / 4.0
    r0, _ = mlp.forward(theta, f)
    r1, s1 = mlp.forward(theta, f, quantize=q)
    if np.array_equal(q(s1["h1"]), s1["h1"]) and np.array_equal(q(np.maximum(s1["z1"], 0)), s1["h1"]):
        assert np.array_equal(r0, r1)
