"""Pins of the classical bicubic comparator (Sec. 5: finite-difference slopes;
Sec. 6: PyTorch's bicubic interpolation) and of the spline upscale at
fractional factors (supplement "Qualitative Results for Different Upsampling
Rates": arbitrary, fractional factors)."""
import numpy as np
import pytest

SIZES = [(7, 5, 14, 10), (6, 9, 18, 27), (10, 6, 15, 9), (7, 5, 11, 8), (13, 11, 20, 17), (4, 4, 4, 4)]


@pytest.mark.parametrize("W,H,W2,H2", SIZES)
def test_bicubic_equals_torch(ora, W, H, W2, H2):
    """a = -0.75 with clamped borders is torch.nn.functional.interpolate(mode
    ='bicubic', align_corners=False), integer and fractional sizes."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(W * 31 + W2)
    C = rng.normal(size=(3, H, W))
    want = torch.nn.functional.interpolate(torch.tensor(C)[None], size=(H2, W2), mode="bicubic",
                                           align_corners=False)[0].numpy()
    got = ora.bicubic(C, W2, H2, a=-0.75)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def _central_grads(C):
    """Central-difference slopes (x, y, xy) on the interior; borders unused."""
    G = np.zeros((3,) + C.shape)
    G[0][:, :, 1:-1] = 0.5 * (C[:, :, 2:] - C[:, :, :-2])
    G[1][:, 1:-1, :] = 0.5 * (C[:, 2:, :] - C[:, :-2, :])
    G[2][:, 1:-1, 1:-1] = 0.25 * (C[:, 2:, 2:] - C[:, 2:, :-2] - C[:, :-2, 2:] + C[:, :-2, :-2])
    return G


@pytest.mark.parametrize("W,H,W2,H2", [(9, 8, 18, 16), (10, 7, 25, 14), (8, 8, 20, 28)])
def test_bicubic_half_is_hermite_with_fd_slopes(ora, W, H, W2, H2):
    """Cubic convolution with a = -1/2 is the Hermite patch whose corner slopes
    are central differences (the classical bicubic of Sec. 5), wherever the 4x4
    samples lie inside the image."""
    rng = np.random.default_rng(5)
    C = rng.normal(size=(3, H, W))
    conv = ora.bicubic(C, W2, H2, a=-0.5)
    herm = ora.upscale(C, _central_grads(C), W2, H2)
    X = np.arange(W2)
    Y = np.arange(H2)
    x = (X + 0.5) * W / W2 - 0.5
    y = (Y + 0.5) * H / H2 - 0.5
    okx = (np.floor(x) >= 1) & (np.floor(x) + 2 <= W - 1)
    oky = (np.floor(y) >= 1) & (np.floor(y) + 2 <= H - 1)
    m = oky[:, None] & okx[None, :]
    assert m.sum() > 20
    np.testing.assert_allclose(conv[:, m], herm[:, m], rtol=0, atol=1e-12)


@pytest.mark.parametrize("a", [-0.5, -0.75])
def test_bicubic_reproduces_constants_and_lines(ora, a):
    """Constants for every a (the weights sum to one); straight lines only for
    a = -1/2, Keys' third-order kernel (other a reproduce constants alone)."""
    W, H, W2, H2 = 9, 7, 21, 16
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    cases = [(np.full((3, H, W), 0.37), True)]
    if a == -0.5:
        cases.append((np.stack([0.1 * xx + 0.05 * yy] * 3), False))
    for C, exact in cases:
        got = ora.bicubic(C, W2, H2, a=a)
        if exact:
            np.testing.assert_allclose(got, 0.37, rtol=0, atol=1e-14)
        else:
            X = (np.arange(W2) + 0.5) * W / W2 - 0.5
            Y = (np.arange(H2) + 0.5) * H / H2 - 0.5
            inner = ((np.floor(Y) >= 1) & (np.floor(Y) + 2 <= H - 1))[:, None] & \
                    ((np.floor(X) >= 1) & (np.floor(X) + 2 <= W - 1))[None, :]
            want = 0.1 * X[None, :] + 0.05 * Y[:, None]
            np.testing.assert_allclose(got[0][inner], np.broadcast_to(want, (H2, W2))[inner], rtol=0, atol=1e-13)


@pytest.mark.parametrize("W,H,W2,H2", [(8, 6, 12, 9), (7, 7, 17, 10), (5, 9, 8, 14)])
def test_spline_fractional_reproduces_cubics(ora, W, H, W2, H2):
    """At fractional factors the Hermite patch still reproduces a bicubic
    polynomial exactly from its values and exact derivatives, borders included."""
    rng = np.random.default_rng(W2)
    A = rng.normal(size=(4, 4))
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)

    def f(x, y, dx=0, dy=0):
        out = np.zeros(np.broadcast(x, y).shape)
        for p in range(4):
            for q in range(4):
                if p < dx or q < dy:
                    continue
                cx = np.prod(range(p - dx + 1, p + 1)) if dx else 1
                cy = np.prod(range(q - dy + 1, q + 1)) if dy else 1
                out = out + A[p, q] * cx * cy * x ** (p - dx) * y ** (q - dy)
        return out

    C = np.stack([f(xx, yy)] * 3)
    G = np.stack([np.stack([f(xx, yy, 1, 0)] * 3), np.stack([f(xx, yy, 0, 1)] * 3),
                  np.stack([f(xx, yy, 1, 1)] * 3)])
    got = ora.upscale(C, G, W2, H2)
    X = (np.arange(W2) + 0.5) * W / W2 - 0.5
    Y = (np.arange(H2) + 0.5) * H / H2 - 0.5
    want = f(X[None, :], Y[:, None])
    np.testing.assert_allclose(got[1], want, rtol=0, atol=1e-9 * np.abs(want).max())
