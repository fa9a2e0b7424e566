"""Pins of the oracle's blend with screen-space derivatives (Sec. 4 blend
equation; Sec. 5 "3DGS Image Gradients"; supplement "Forward pass").

Independent references: sympy differentiates the closed form
I = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j) symbolically; finite differences
of the oracle's own image in screen space; invariants of uniform colour; and the
decision rules of the 3DGS mode on configurations whose result is known by hand.
"""
import numpy as np
import pytest
import sympy as sp

import scenes


def make_2d(ora, means, conics, ops, cols, depths, W, H, mode, tile=16):
    """A projected-scene dict built by hand (bypasses projection); every Gaussian
    is binned into every tile so binning cannot drop a contribution."""
    n = len(means)
    tx, ty = (W + tile - 1) // tile, (H + tile - 1) // tile
    proj = dict(mean2d=np.asarray(means, float).reshape(n, 2),
                conic=np.asarray(conics, float).reshape(n, 3),
                opacity=np.asarray(ops, float).reshape(n),
                rgb=np.asarray(cols, float).reshape(n, 3),
                depth=np.asarray(depths, float).reshape(n),
                rect=np.tile(np.array([0, 0, tx - 1, ty - 1], np.int32), (n, 1)),
                tiles_touched=np.full(n, tx * ty, np.int64),
                W=W, H=H, tile=tile, mode=mode, tiles_x=tx, tiles_y=ty)
    return proj, ora.bin_pairs(proj)


def random_2d(rng, n, W, H):
    means = np.stack([rng.uniform(-2, W + 1, n), rng.uniform(-2, H + 1, n)], 1)
    conics = []
    for _ in range(n):
        L = rng.normal(0, 1, (2, 2))
        cov = L @ L.T * rng.uniform(2, 12) + 0.5 * np.eye(2)
        Q = np.linalg.inv(cov)
        conics.append([Q[0, 0], Q[0, 1], Q[1, 1]])
    ops = rng.uniform(0.2, 0.95, n)
    cols = rng.uniform(0, 1, (n, 3))
    depths = rng.uniform(1, 5, n)
    return means, np.array(conics), ops, cols, depths


def sympy_image(means, conics, ops, cols, depths, bg):
    """Closed-form I(x, y) and its derivatives, sorted front to back."""
    x, y = sp.symbols("x y", real=True)
    order = sorted(range(len(means)), key=lambda i: (np.float32(depths[i]), i))
    exprs = []
    for ch in range(3):
        I = 0
        trans = 1
        for i in order:
            dx, dy = x - means[i][0], y - means[i][1]
            a, b, c = conics[i]
            alpha = ops[i] * sp.exp(-sp.Rational(1, 2) * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
            I += cols[i][ch] * alpha * trans
            trans *= (1 - alpha)
        I += bg[ch] * trans
        exprs.append([I, sp.diff(I, x), sp.diff(I, y), sp.diff(I, x, y)])
    fns = [[sp.lambdify((x, y), e, "numpy") for e in row] for row in exprs]
    return fns


@pytest.mark.parametrize("n,bg", [(1, (0, 0, 0)), (2, (0, 0, 0)), (4, (0.2, 0.5, 0.9))])
def test_exact_mode_matches_symbolic(ora, n, bg):
    W, H = 20, 18
    rng = np.random.default_rng(n)
    means, conics, ops, cols, depths = random_2d(rng, n, W, H)
    means[:, 0] = rng.uniform(4, 16, n)
    means[:, 1] = rng.uniform(4, 14, n)
    proj, bins = make_2d(ora, means, conics, ops, cols, depths, W, H, ora.MODE_EXACT)
    res = ora.render(proj, bins, bg=bg)
    fns = sympy_image(means, conics, ops, cols, depths, bg)
    Y, X = np.mgrid[0:H, 0:W].astype(float)
    for ch in range(3):
        want = [np.broadcast_to(f(X, Y), (H, W)) for f in fns[ch]]
        np.testing.assert_allclose(res["C"][ch], want[0], rtol=1e-12, atol=1e-13)
        for k in range(3):
            np.testing.assert_allclose(res["grads"][k, ch], want[k + 1], rtol=1e-10, atol=1e-12)


def test_single_gaussian_closed_form(ora):
    """T = 1: C = c alpha, C_x = c alpha g_x, C_y = c alpha g_y,
    C_xy = c alpha (g_x g_y + g_xy) with g = -1/2 d^T Q d."""
    W, H = 16, 16
    m = np.array([[7.3, 8.6]])
    Qc = np.array([[0.3, 0.1, 0.5]])
    op, col = np.array([0.8]), np.array([[0.25, 0.5, 1.0]])
    proj, bins = make_2d(ora, m, Qc, op, col, [2.0], W, H, ora.MODE_EXACT)
    res = ora.render(proj, bins)
    Y, X = np.mgrid[0:H, 0:W].astype(float)
    dx, dy = X - 7.3, Y - 8.6
    a, b, c = 0.3, 0.1, 0.5
    g = -0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy)
    gx, gy, gxy = -(a * dx + b * dy), -(b * dx + c * dy), -b
    al = 0.8 * np.exp(g)
    for ch in range(3):
        np.testing.assert_allclose(res["C"][ch], col[0, ch] * al, rtol=1e-13, atol=1e-16)
        np.testing.assert_allclose(res["grads"][0, ch], col[0, ch] * al * gx, rtol=1e-12, atol=1e-16)
        np.testing.assert_allclose(res["grads"][1, ch], col[0, ch] * al * gy, rtol=1e-12, atol=1e-16)
        np.testing.assert_allclose(res["grads"][2, ch], col[0, ch] * al * (gx * gy + gxy), rtol=1e-11, atol=1e-15)


def test_uniform_colour_invariant(ora):
    """All c_i = c: C = c A_N and each derivative of C is c times that of A_N."""
    W, H = 24, 20
    rng = np.random.default_rng(11)
    n = 9
    means, conics, ops, cols, depths = random_2d(rng, n, W, H)
    cols[:] = [0.3, 0.6, 0.9]
    for mode in (ora.MODE_EXACT, ora.MODE_3DGS):
        proj, bins = make_2d(ora, means, conics, ops, cols, depths, W, H, mode)
        res = ora.render(proj, bins)
        st = res["state"]
        for ch in range(3):
            c = cols[0, ch]
            np.testing.assert_allclose(res["C"][ch], c * st[0], rtol=1e-12, atol=1e-15)
            for k in range(3):
                np.testing.assert_allclose(res["grads"][k, ch], c * st[k + 1], rtol=1e-10, atol=1e-14)


def test_screen_space_finite_differences(ora):
    """Shifting the evaluation grid by +-h: central differences of C match the
    analytic C_x, C_y; the four-point stencil matches C_xy."""
    W, H = 32, 32
    scene = scenes.random_scene(60, seed=4, xy_range=0.6, log_scale_mean=-2.5)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H, mode=ora.MODE_EXACT)
    bins = ora.bin_pairs(proj)
    base = ora.render(proj, bins)
    h = 1e-4

    def C_at(ox, oy):
        return ora.render(proj, bins, offset=(ox, oy))["C"]

    fdx = (C_at(h, 0) - C_at(-h, 0)) / (2 * h)
    fdy = (C_at(0, h) - C_at(0, -h)) / (2 * h)
    fdxy = (C_at(h, h) - C_at(h, -h) - C_at(-h, h) + C_at(-h, -h)) / (4 * h * h)
    scale = [np.abs(base["grads"][k]).max() for k in range(3)]
    np.testing.assert_allclose(fdx, base["grads"][0], atol=2e-6 * scale[0])
    np.testing.assert_allclose(fdy, base["grads"][1], atol=2e-6 * scale[1])
    np.testing.assert_allclose(fdxy, base["grads"][2], atol=2e-4 * scale[2])


def test_3dgs_cutoff_skips_faint_gaussians(ora):
    """Opacity below 1/255: alpha < 1/255 everywhere, the Gaussian never blends."""
    W, H = 16, 16
    means = [[8, 8], [8, 8]]
    conics = [[0.2, 0, 0.2], [0.1, 0, 0.1]]
    proj, bins = make_2d(ora, means, conics, [0.003, 0.5], [[1, 1, 1], [0.2, 0.4, 0.6]], [1.0, 2.0],
                         W, H, ora.MODE_3DGS)
    res = ora.render(proj, bins)
    proj2, bins2 = make_2d(ora, means[1:], conics[1:], [0.5], [[0.2, 0.4, 0.6]], [2.0], W, H, ora.MODE_3DGS)
    res2 = ora.render(proj2, bins2)
    np.testing.assert_array_equal(res["C"], res2["C"])
    np.testing.assert_array_equal(res["grads"], res2["grads"])


def test_3dgs_termination_count(ora):
    """Ten identical Gaussians of opacity 0.85 centred on a pixel: transmittance
    after k of them is 0.15^k; the pixel stops before the fifth (0.15^5 < 1e-4),
    so exactly four blend and C = c (1 - 0.15^4) there."""
    W, H = 16, 16
    n = 10
    means = [[5.0, 6.0]] * n
    conics = [[0.05, 0.0, 0.05]] * n
    cols = [[0.5, 0.25, 1.0]] * n
    proj, bins = make_2d(ora, means, conics, [0.85] * n, cols, np.arange(1, n + 1, dtype=float), W, H,
                         ora.MODE_3DGS)
    res = ora.render(proj, bins)
    assert res["state"][4, 6, 5] == 4
    np.testing.assert_allclose(res["C"][:, 6, 5], np.array(cols[0]) * (1 - 0.15 ** 4), rtol=1e-14)


def test_3dgs_clamp_zeroes_alpha_derivatives(ora):
    """Opacity 1 at the centre: alpha = min(0.99, 1) is constant, so the mixed
    derivative there is 0 (it is c alpha (-b) != 0 without the clamp)."""
    W, H = 16, 16
    proj, bins = make_2d(ora, [[5.0, 6.0]], [[0.3, 0.2, 0.4]], [1.0], [[1.0, 1.0, 1.0]], [1.0], W, H,
                         ora.MODE_3DGS)
    res = ora.render(proj, bins)
    np.testing.assert_allclose(res["C"][:, 6, 5], 0.99, rtol=1e-15)
    assert np.all(res["grads"][:, :, 6, 5] == 0.0)
    proj, bins = make_2d(ora, [[5.0, 6.0]], [[0.3, 0.2, 0.4]], [1.0], [[1.0, 1.0, 1.0]], [1.0], W, H,
                         ora.MODE_EXACT)
    res = ora.render(proj, bins)
    np.testing.assert_allclose(res["grads"][2, :, 6, 5], -0.2, rtol=1e-14)


def test_variant_zero_is_nominal(ora):
    W, H = 64, 64
    scene = scenes.random_scene(1000, seed=0)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    bins = ora.bin_pairs(proj)
    res = ora.render(proj, bins, variants=True)
    v0 = res["variants"][:, :, 0, :].transpose(2, 0, 1)
    np.testing.assert_array_equal(v0[0:3], res["C"])
    np.testing.assert_array_equal(v0[3:12].reshape(3, 3, H, W), res["grads"])
    assert (res["nvar"] >= 1).mean() > 0.98


def test_sampled_pixels_match_full(ora):
    W, H = 40, 30
    scene = scenes.random_scene(300, seed=2)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    bins = ora.bin_pairs(proj)
    full = ora.render(proj, bins)
    rng = np.random.default_rng(0)
    pix = np.stack([rng.integers(0, W, 64), rng.integers(0, H, 64)], 1)
    samp = ora.render(proj, bins, pixels=pix)
    np.testing.assert_array_equal(samp["out"][:, 0:3], full["C"][:, pix[:, 1], pix[:, 0]].T)
    np.testing.assert_array_equal(samp["out"][:, 3:6], full["grads"][0][:, pix[:, 1], pix[:, 0]].T)


def test_analytic_slopes_beat_finite_differences(ora):
    """The paper's motivation (Sec. 3, and Bicubic vs Spline in Table 1): the
    Hermite patch with analytic image gradients reconstructs the continuous
    low-res image between pixels better than with finite-difference slopes."""
    W, H, s = 32, 32, 4
    scene = scenes.random_scene(80, seed=9, xy_range=0.6, log_scale_mean=-2.8)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H, mode=ora.MODE_EXACT)
    bins = ora.bin_pairs(proj)
    base = ora.render(proj, bins)
    # ground truth: the continuous image at every hi-res sample point x = (X + 0.5)/s - 0.5
    truth = np.zeros((3, s * H, s * W))
    for a in range(s):
        for b in range(s):
            ox, oy = (a + 0.5) / s - 0.5, (b + 0.5) / s - 0.5
            C = ora.render(proj, bins, offset=(ox, oy))["C"]
            # hi-res X = s * i + a samples low-res point i + ox
            truth[:, b::s, a::s] = C
    spline = ora.upscale(base["C"], base["grads"], s * W, s * H)
    C = base["C"]
    fd = np.zeros_like(base["grads"])
    fd[0] = np.gradient(C, axis=2)
    fd[1] = np.gradient(C, axis=1)
    fd[2] = np.gradient(fd[0], axis=1)
    bicubic = ora.upscale(C, fd, s * W, s * H)
    inner = (slice(None), slice(s, -s), slice(s, -s))
    err_a = np.sqrt(np.mean((spline - truth)[inner] ** 2))
    err_f = np.sqrt(np.mean((bicubic - truth)[inner] ** 2))
    assert err_a < 0.7 * err_f, (err_a, err_f)
