"""FP64 oracle of the learned residual on top of the spline upscale.

TEST INFRASTRUCTURE ONLY (like the rest of this package): called by the tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference leg,
never by the product path.

The paper upscales with the gradient-aware Hermite spline alone (Sec. 5) and
argues against learned upscalers (Sec. 2).  This module defines the optional
learned part that sits on top of it: a per-output-pixel MLP that reads the same
48 values the spline reads and adds a residual.  The definition is written out
plainly:

  features f (50 per output pixel, in this order):
      f[12 k + 3 q + c]   corner k of the pixel's spline cell (k = 0: (i, j),
                          1: (i+1, j), 2: (i, j+1), 3: (i+1, j+1)), quantity q
                          (0: C, 1: dC/dx, 2: dC/dy, 3: d2C/dxdy), channel c
      f[48], f[49]        the local coordinates t, u of the sample point in the
                          cell (the spline's own, Sec. 5; outside [0, 1] in the
                          border half-cells)
  h1 = relu(W1 f + b1)        W1 [64, 50], b1 [64]
  h2 = relu(W2 h1 + b2)       W2 [64, 64], b2 [64]
  r  = W3 h2 + b3             W3 [3, 64],  b3 [3]
  out = spline(X, Y) + r

The cell of output pixel X of a W2-wide image is i = clamp(floor(x), 0, W - 2)
with x = (X + 0.5) W / W2 - 0.5 and t = x - i, as for the spline.

Parameters travel as one flat vector in the order W1, b1, W2, b2, W3, b3 (row
major), 7619 values.  The training loss is the mean squared error over samples
and channels, L = sum (out - target)^2 / (3 M), and the optimiser is Adam
(Kingma and Ba, 2015) with bias correction.
"""
from __future__ import annotations

import numpy as np

N_IN = 50
N_HID = 64
N_OUT = 3
SHAPES = (("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta) -> dict:
    """Flat parameter vector -> dict of arrays (views)."""
    theta = np.asarray(theta, np.float64)
    assert theta.shape == (N_PARAMS,)
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[k:k + n].reshape(shape)
        k += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], np.float64).reshape(-1) for name, _ in SHAPES])


def cells(X, W: int, W2: int):
    """Cell index i = clamp(floor(x), 0, W - 2) and t = x - i for output
    columns X, x = (X + 0.5) W / W2 - 0.5 (the spline's half-pixel map)."""
    X = np.asarray(X, np.int64)
    x = (X + 0.5) * W / W2 - 0.5
    i = np.clip(np.floor(x).astype(np.int64), 0, W - 2)
    return i, x - i


def features(C, grads, W2: int, H2: int, pixels=None) -> np.ndarray:
    """The 50 inputs of each output pixel: [M, 50] for pixels [M, 2] of (X, Y),
    or [H2 * W2, 50] in row-major pixel order for pixels=None."""
    C = np.asarray(C, np.float64)
    G = np.asarray(grads, np.float64)
    H, W = C.shape[1:]
    if pixels is None:
        Y, X = np.divmod(np.arange(W2 * H2), W2)
    else:
        pix = np.asarray(pixels, np.int64).reshape(-1, 2)
        X, Y = pix[:, 0], pix[:, 1]
    i, t = cells(X, W, W2)
    j, u = cells(Y, H, H2)
    planes = (C, G[0], G[1], G[2])           # C, dC/dx, dC/dy, d2C/dxdy; each [3, H, W]
    f = np.zeros((len(X), N_IN))
    for k, (di, dj) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
        for q in range(4):
            for c in range(3):
                f[:, 12 * k + 3 * q + c] = planes[q][c, j + dj, i + di]
    f[:, 48] = t
    f[:, 49] = u
    return f


def forward(theta, f, quantize=None):
    """MLP residual r [M, 3] of features f [M, 50], with the intermediates.

    ``quantize`` (e.g. ``bf16_round``), when given, is applied where a lower-
    precision evaluation stores an operand in a narrower type: to the features,
    to h1 before the second layer and to h2 before the output layer.  That
    rounding is a quantisation decision (the code of the narrow value), taken
    here on this definition's values."""
    p = unpack(theta)
    f = np.asarray(f, np.float64)
    if quantize is not None:
        f = quantize(f)
    z1 = f @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    if quantize is not None:
        h1 = quantize(h1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    if quantize is not None:
        h2 = quantize(h2)
    r = h2 @ p["W3"].T + p["b3"]
    return r, dict(z1=z1, h1=h1, z2=z2, h2=h2)


def upscale(C, grads, W2: int, H2: int, theta, pixels=None) -> np.ndarray:
    """Spline plus residual: [3, H2, W2] (pixels=None) or [M, 3]."""
    from . import upscale as spline_upscale
    f = features(C, grads, W2, H2, pixels)
    r, _ = forward(theta, f)
    base = spline_upscale(C, grads, W2, H2, pixels=pixels)
    if pixels is None:
        return base + r.T.reshape(3, H2, W2)
    return base + r


def loss(theta, f, base, target) -> float:
    """L = sum over samples and channels of (base + r - target)^2 / (3 M)."""
    r, _ = forward(theta, f)
    e = np.asarray(base, np.float64) + r - np.asarray(target, np.float64)
    return float(np.sum(e * e) / e.size)


def gradient(theta, f, base, target, masks=None, quantize=None):
    """dL/dtheta (flat, the order of ``pack``) by reverse-mode chain rule, and L.

    The ReLU derivative is 1 where z > 0, else 0.  ``masks`` = (z1 > 0, z2 > 0)
    as boolean [M, 64] arrays replaces those decisions when given, and
    ``quantize`` is applied as in ``forward`` and to d2 and d1 before they are
    multiplied (the points where a lower-precision evaluation narrows them)."""
    p = unpack(theta)
    q = (lambda a: a) if quantize is None else quantize
    f = q(np.asarray(f, np.float64))
    r, s = forward(theta, f, quantize)
    m1, m2 = (s["z1"] > 0, s["z2"] > 0) if masks is None else masks
    e = np.asarray(base, np.float64) + r - np.asarray(target, np.float64)
    d3 = 2.0 * e / e.size                        # dL/dr            [M, 3]
    g = {"W3": d3.T @ s["h2"], "b3": d3.sum(0)}
    d2 = q((d3 @ p["W3"]) * m2)                  # dL/dz2           [M, 64]
    g["W2"] = d2.T @ s["h1"]
    g["b2"] = d2.sum(0)
    d1 = q((d2 @ p["W2"]) * m1)                  # dL/dz1           [M, 64]
    g["W1"] = d1.T @ f
    g["b1"] = d1.sum(0)
    return pack(g), float(np.sum(e * e) / e.size)


def adam(theta, m, v, g, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1) at step >= 1:
    returns the new (theta, m, v)."""
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return np.asarray(theta, np.float64) - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a) -> np.ndarray:
    """Round to the nearest bfloat16 value (ties to even), returned as float64.
    bfloat16 keeps the sign, the 8 exponent bits and the top 7 mantissa bits of
    an IEEE binary32; rounding adds half of the dropped range (0x7FFF plus the
    kept least significant bit, for ties to even) before truncating."""
    b = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    r = ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r.astype(np.uint32)).view(np.float32).astype(np.float64)
