"""Comparing the tensor-core MLP kernels with the FP64 oracle (oracle.mlp).

The kernels narrow operands to BF16 (8 significant bits) at fixed points: the
matrices, the features, h1 before the second layer, h2 before the output
layer, d2 and d1 before the reverse-mode products.  Each narrowing is a quantisation decision, so the
reference takes it in the kernels' precision: oracle.mlp evaluated with
``quantize = bf16_round`` on the BF16 values of the matrices.  What remains
between kernel and reference is FP32 accumulation, bounded as follows:

  * a sum of n terms with exact products (BF16 x BF16 products are exact in
    FP32) carries at most n G sum |terms|, G = 2^-23 (the FP32 unit roundoff
    doubled, which also covers accumulators that truncate);
  * the long sums over samples of the weight gradients use the probabilistic
    bound of Higham and Mary (SIAM J. Sci. Comput. 2019), lambda sqrt(n) G
    times the sum of |terms|, with lambda = 8;
  * a value within its accumulation bound of a BF16 rounding boundary (the
    midpoint of consecutive BF16 values) may round the other way in the kernel:
    one BF16 step, propagated through the absolute weights;
  * ReLU derivative decisions whose z lies within its bound of 0 are ambiguous;
    samples with one are dropped from the comparison.
"""
from __future__ import annotations

import numpy as np

from oracle import mlp

U = 2.0 ** -8      # BF16 unit roundoff
G = 2.0 ** -23     # FP32 unit roundoff, doubled
LAMBDA = 8.0

q = mlp.bf16_round


def bf16_params(theta):
    """theta with W1, W2, W3 rounded to BF16 values (biases unchanged)."""
    p = {k: np.array(v) for k, v in mlp.unpack(theta).items()}
    for k in ("W1", "W2", "W3"):
        p[k] = q(p[k])
    return mlp.pack(p)


def ulp(x):
    """Spacing of BF16 values at |x| (0 at 0)."""
    a = np.abs(np.asarray(x, np.float64))
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    return np.where(a > 0, 2.0 ** (e - 7), 0.0)


def flip_step(x, e):
    """One BF16 step where a value within e of x may round differently from x:
    x within e of a rounding boundary; else 0."""
    x = np.asarray(x, np.float64)
    r = q(x)
    u = np.maximum(ulp(x), ulp(r))
    return np.where(0.5 * u - np.abs(x - r) <= e, u, 0.0)


def forward_reference(theta_b, f):
    """Reference residual (kernel precision), its bound per sample and channel,
    and the samples whose ReLU decisions are unambiguous."""
    p = mlp.unpack(theta_b)
    A1, A2, A3 = np.abs(p["W1"]), np.abs(p["W2"]), np.abs(p["W3"])
    r, s = mlp.forward(theta_b, f, quantize=q)
    fq = q(np.asarray(f, np.float64))
    e1 = 64 * G * (np.abs(fq) @ A1.T + np.abs(p["b1"]))
    # h1 before rounding (relu of the FP64 z1) and the rounding it may take
    h1_pre = np.maximum(s["z1"], 0.0)
    eh1 = flip_step(h1_pre, e1)
    e2 = eh1 @ A2.T + 66 * G * (s["h1"] @ A2.T + np.abs(p["b2"]))
    h2_pre = np.maximum(s["z2"], 0.0)
    eh2 = flip_step(h2_pre, e2)
    e3 = eh2 @ A3.T + 66 * G * (s["h2"] @ A3.T + np.abs(p["b3"]))
    keep = np.all(np.abs(s["z1"]) > 2 * e1, axis=1) & np.all(np.abs(s["z2"]) > 2 * e2, axis=1)
    return dict(r=r, e3=e3, keep=keep, e1=e1, e2=e2, eh1=eh1, eh2=eh2, **s)


def gradient_reference(theta_b, f, base, target):
    """Reference gradient (kernel precision) with its elementwise bound and the
    loss with its bound.  f must hold BF16 values; samples with ambiguous ReLU
    decisions must have been dropped (forward_reference's keep)."""
    p = mlp.unpack(theta_b)
    A2, A3 = np.abs(p["W2"]), np.abs(p["W3"])
    fw = forward_reference(theta_b, f)
    assert fw["keep"].all()
    M = f.shape[0]
    base = np.asarray(base, np.float64)
    target = np.asarray(target, np.float64)
    m1, m2 = fw["z1"] > 0, fw["z2"] > 0
    g, L = mlp.gradient(theta_b, f, base, target, quantize=q)
    r, h1, h2 = fw["r"], fw["h1"], fw["h2"]
    e = base + r - target
    ee = fw["e3"] + 3 * G * (np.abs(base) + np.abs(r) + np.abs(target))
    d3 = 2.0 * e / e.size
    ed3 = 2.0 * ee / e.size + 2 * G * np.abs(d3)
    d2 = (d3 @ p["W3"]) * m2
    ed2 = (ed3 @ A3 + 3 * G * (np.abs(d3) @ A3)) * m2
    ed2q = flip_step(d2, ed2)
    d2q = q(d2)
    d1 = (d2q @ p["W2"]) * m1
    ed1 = (ed2q @ A2 + 64 * G * (np.abs(d2q) @ A2)) * m1
    ed1q = flip_step(d1, ed1)
    d1q = q(d1)
    eh1 = fw["eh1"]
    eh2 = fw["eh2"]
    fa = np.abs(np.asarray(f, np.float64))
    acc = LAMBDA * np.sqrt(M) * G          # the sums over samples
    bound = {
        "W3": ed3.T @ (h2 + eh2) + np.abs(d3).T @ eh2 + acc * (np.abs(d3).T @ h2),
        "b3": ed3.sum(0) + acc * np.abs(d3).sum(0),
        "W2": ed2q.T @ (h1 + eh1) + np.abs(d2q).T @ eh1 + acc * (np.abs(d2q).T @ h1),
        "b2": ed2q.sum(0) + acc * np.abs(d2q).sum(0),
        "W1": ed1q.T @ fa + acc * (np.abs(d1q).T @ fa),
        "b1": ed1q.sum(0) + acc * np.abs(d1q).sum(0),
    }
    eL = float(np.sum(2 * np.abs(e) * ee + ee * ee) / e.size + acc * np.sum(e * e) / e.size)
    return g, mlp.pack(bound), L, eL


def random_theta(rng, scale=(0.25, 0.2, 0.3), bias=0.1):
    p = {"W1": rng.normal(0, scale[0], (64, 50)), "b1": rng.normal(0, bias, 64),
         "W2": rng.normal(0, scale[1], (64, 64)), "b2": rng.normal(0, bias, 64),
         "W3": rng.normal(0, scale[2], (3, 64)), "b3": rng.normal(0, bias, 3)}
    return mlp.pack(p)
