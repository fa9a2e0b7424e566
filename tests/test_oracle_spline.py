"""Pins of the oracle's spline upscale (Sec. 5 "Spline Interpolation"; supplement
"Spline Image Interpolation") against facts that do not come from the oracle:
the printed matrix C, the textbook cubic Hermite basis, exact reproduction of
bicubic polynomials, and the interpolation property."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hermite_C.txt")


def _golden_C():
    return np.loadtxt(GOLDEN, comments="#")


def test_cinv_inverts_printed_C(ora):
    C = _golden_C()
    Ci = ora.spline_cinv()
    np.testing.assert_allclose(C @ Ci, np.eye(4), atol=1e-15)
    np.testing.assert_allclose(Ci @ C, np.eye(4), atol=1e-15)


def test_basis_is_cubic_hermite(ora):
    """[1 t t^2 t^3] C^-1 must be the textbook Hermite basis (h00, h01, h10, h11)."""
    Ci = ora.spline_cinv()
    for t in np.linspace(-0.6, 1.6, 23):
        row = np.array([1.0, t, t * t, t ** 3]) @ Ci
        h00 = 2 * t ** 3 - 3 * t ** 2 + 1
        h01 = -2 * t ** 3 + 3 * t ** 2
        h10 = t ** 3 - 2 * t ** 2 + t
        h11 = t ** 3 - t ** 2
        np.testing.assert_allclose(row, [h00, h01, h10, h11], atol=1e-14)


def _poly_image(coef, W, H):
    """f(x, y) = sum a_ij x^i y^j on the low-res grid (x = column, y = row) with
    its exact first and mixed derivatives."""
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    xs = xs / W
    ys = ys / H

    def ev(dx, dy):
        out = np.zeros((H, W))
        for i in range(4):
            for j in range(4):
                if i < dx or j < dy:
                    continue
                ci = np.prod(range(i - dx + 1, i + 1)) if dx else 1.0
                cj = np.prod(range(j - dy + 1, j + 1)) if dy else 1.0
                out += coef[i, j] * ci * cj * xs ** (i - dx) * ys ** (j - dy)
        return out / (W ** dx) / (H ** dy)

    return ev(0, 0), ev(1, 0), ev(0, 1), ev(1, 1)


def _poly_at(coef, x, y, W, H):
    xs, ys = x / W, y / H
    return sum(coef[i, j] * xs ** i * ys ** j for i in range(4) for j in range(4))


@pytest.mark.parametrize("W,H,s", [(7, 5, 1), (7, 5, 2), (9, 6, 3), (6, 7, 4), (5, 4, 8), (13, 3, 2)])
def test_reproduces_bicubic_polynomials(ora, W, H, s):
    """A cubic Hermite patch is exact for bicubic data: every output, interior
    and extrapolated border, equals f at the hi-res sample point."""
    rng = np.random.default_rng(W * 100 + H * 10 + s)
    coefs = rng.normal(0, 1, (3, 4, 4))
    C = np.zeros((3, H, W))
    G = np.zeros((3, 3, H, W))
    for ch in range(3):
        f, fx, fy, fxy = _poly_image(coefs[ch], W, H)
        C[ch], G[0, ch], G[1, ch], G[2, ch] = f, fx, fy, fxy
    W2, H2 = s * W, s * H
    out = ora.upscale(C, G, W2, H2)
    Y, X = np.mgrid[0:H2, 0:W2].astype(np.float64)
    x = (X + 0.5) / s - 0.5
    y = (Y + 0.5) / s - 0.5
    for ch in range(3):
        want = _poly_at(coefs[ch], x, y, W, H)
        np.testing.assert_allclose(out[ch], want, rtol=0, atol=1e-10 * (1 + np.abs(want).max()))


def test_transposed_derivatives_are_caught(ora):
    """Sanity of the pin above: swapping f_x and f_y breaks reproduction."""
    W, H = 8, 6
    coef = np.zeros((4, 4))
    coef[3, 0] = 1.0      # f = x^3 depends on x only
    f, fx, fy, fxy = _poly_image(coef, W, H)
    C = np.stack([f] * 3)
    G = np.stack([np.stack([fy] * 3), np.stack([fx] * 3), np.stack([fxy] * 3)])
    out = ora.upscale(C, G, 2 * W, 2 * H)
    Y, X = np.mgrid[0:2 * H, 0:2 * W].astype(np.float64)
    want = _poly_at(coef, (X + 0.5) / 2 - 0.5, (Y + 0.5) / 2 - 0.5, W, H)
    assert np.abs(out[0] - want).max() > 1e-4


@pytest.mark.parametrize("s", [1, 3, 5])
def test_interpolation_property(ora, s):
    """Where a hi-res sample lands on a low-res pixel (t = u = 0) the output is
    that pixel's value, bit for bit; on-grid samples at t = 1 agree to rounding."""
    W, H = 6, 5
    rng = np.random.default_rng(s)
    C = rng.uniform(0, 1, (3, H, W))
    G = rng.normal(0, 1, (3, 3, H, W))
    out = ora.upscale(C, G, s * W, s * H)
    off = (s - 1) // 2
    for j in range(H):
        for i in range(W):
            X, Y = s * i + off, s * j + off
            if i < W - 1 and j < H - 1:
                assert np.array_equal(out[:, Y, X], C[:, j, i])
            else:
                np.testing.assert_allclose(out[:, Y, X], C[:, j, i], atol=1e-13)


def test_factor_one_is_identity(ora):
    W, H = 9, 7
    rng = np.random.default_rng(3)
    C = rng.uniform(0, 1, (3, H, W))
    G = rng.normal(0, 1, (3, 3, H, W))
    out = ora.upscale(C, G, W, H)
    np.testing.assert_allclose(out, C, atol=1e-13)


def test_sampled_matches_full(ora):
    W, H, s = 10, 7, 4
    rng = np.random.default_rng(5)
    C = rng.uniform(0, 1, (3, H, W))
    G = rng.normal(0, 1, (3, 3, H, W))
    full = ora.upscale(C, G, s * W, s * H)
    pix = np.stack([rng.integers(0, s * W, 50), rng.integers(0, s * H, 50)], 1)
    samp = ora.upscale(C, G, s * W, s * H, pixels=pix)
    np.testing.assert_array_equal(samp, full[:, pix[:, 1], pix[:, 0]].T)


def test_upscale_rejects_degenerate(ora):
    with pytest.raises(ValueError):
        ora.upscale(np.zeros((3, 1, 5)), np.zeros((3, 3, 1, 5)), 10, 2)
