"""Pins of the oracle's reverse mode (supplement "Backward Pass") against facts
that do not come from the oracle's own adjoint code: the adjoint identity of a
linear map, the front-to-back = back-to-front identity of the blend, and FP64
central finite differences of the oracle's forward functions."""
import numpy as np
import pytest

import scenes


def _dot(a, b):
    return float(np.sum(np.asarray(a, np.float64) * np.asarray(b, np.float64)))


# ---------------------------------------------------------------- upscale

@pytest.mark.parametrize("W,H,W2,H2", [(7, 5, 14, 10), (6, 9, 18, 27), (5, 4, 13, 9), (2, 2, 8, 8)])
def test_upscale_adjoint_identity(ora, W, H, W2, H2):
    """<dout, U v> = <U^T dout, v> for random v and dout (U linear)."""
    rng = np.random.default_rng(W * 100 + H2)
    C = rng.normal(size=(3, H, W))
    G = rng.normal(size=(3, 3, H, W))
    dout = rng.normal(size=(3, H2, W2))
    lhs = _dot(dout, ora.upscale(C, G, W2, H2))
    dC, dG = ora.upscale_adjoint(dout, W, H)
    rhs = _dot(dC, C) + _dot(dG, G)
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + np.abs(dout).sum())


def test_upscale_adjoint_unit_columns(ora):
    """Each low-res value's adjoint equals the upscale of that unit input
    contracted with dout (the definition of the transpose, by columns)."""
    rng = np.random.default_rng(3)
    W, H, s = 4, 3, 3
    dout = rng.normal(size=(3, H * s, W * s))
    dC, dG = ora.upscale_adjoint(dout, W, H)
    for q in range(12):
        for (y, x) in [(0, 0), (1, 2), (2, 3)]:
            C = np.zeros((3, H, W))
            G = np.zeros((3, 3, H, W))
            ch = q % 3
            if q < 3:
                C[ch, y, x] = 1.0
                want = dC[ch, y, x]
            else:
                G[q // 3 - 1, ch, y, x] = 1.0
                want = dG[q // 3 - 1, ch, y, x]
            assert abs(_dot(dout, ora.upscale(C, G, W * s, H * s)) - want) < 1e-12


# ---------------------------------------------------------------- blend

def _small(ora, mode, n=40, W=32, H=24, seed=1, bg=(0.2, 0.4, 0.1), sh=None):
    scene = scenes.random_scene(n=n, seed=seed, sh_degree=sh, log_scale_mean=-2.2, xy_range=0.7)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H, mode=mode)
    bins = ora.bin_pairs(proj)
    return scene, cam, proj, bins


@pytest.mark.parametrize("mode", [0, 1])
def test_back_to_front_equals_front_to_back(ora, mode):
    """B^_1 of the backward recurrence (background as B^_{N+1}) and its x, y, xy
    derivatives equal the forward A/B recurrences' image."""
    bg = (0.2, 0.4, 0.1)
    _, _, proj, bins = _small(ora, mode, n=200, bg=bg)
    fwd = ora.render(proj, bins, bg=bg)
    W, H = proj["W"], proj["H"]
    rng = np.random.default_rng(0)
    r = ora.render_adjoint(proj, bins, (rng.normal(size=(3, H, W)), rng.normal(size=(3, 3, H, W))), bg=bg)
    np.testing.assert_allclose(r["b2f_C"], fwd["C"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r["b2f_grads"], fwd["grads"], rtol=0, atol=1e-11 * (1 + np.abs(fwd["grads"]).max()))


def _loss_render(ora, proj, bins, u, bg):
    r = ora.render(proj, bins, bg=bg)
    return _dot(u[0], r["C"]) + _dot(u[1], r["grads"])


FIELD = {0: ("mean2d", 0), 1: ("mean2d", 1), 2: ("conic", 0), 3: ("conic", 1), 4: ("conic", 2),
         5: ("opacity", None), 6: ("rgb", 0), 7: ("rgb", 1), 8: ("rgb", 2)}


def _perturbed(proj, i, f, h):
    key, col = FIELD[f]
    p2 = dict(proj)
    p2[key] = proj[key].copy()
    if col is None:
        p2[key][i] += h
    else:
        p2[key][i, col] += h
    return p2


def test_render_adjoint_fd_exact(ora):
    """Exact mode (smooth in every 2D parameter): analytic gradients of
    L = <u, (C, C_x, C_y, C_xy)> equal FP64 central differences."""
    bg = (0.2, 0.4, 0.1)
    _, _, proj, bins = _small(ora, 1, n=30)
    W, H = proj["W"], proj["H"]
    rng = np.random.default_rng(5)
    u = (rng.normal(size=(3, H, W)), rng.normal(size=(3, 3, H, W)))
    g = ora.render_adjoint(proj, bins, u, bg=bg)["g2d"]
    vis = np.flatnonzero(proj["radius"] > 0)
    assert vis.size >= 10
    for i in vis[:10]:
        for f in range(9):
            val = proj[FIELD[f][0]][i] if FIELD[f][1] is None else proj[FIELD[f][0]][i, FIELD[f][1]]
            h = 1e-6 * max(1.0, abs(val))
            fd = (_loss_render(ora, _perturbed(proj, i, f, h), bins, u, bg) -
                  _loss_render(ora, _perturbed(proj, i, f, -h), bins, u, bg)) / (2 * h)
            assert abs(fd - g[i, f]) <= 2e-6 * (abs(fd) + 1e-3 * np.abs(g).max()), (i, f, fd, g[i, f])


def test_render_adjoint_fd_3dgs(ora):
    """3dgs mode: where a perturbation flips no decision (same blended pairs and
    stops on both sides), the gradient equals the central difference."""
    bg = (0.0, 0.0, 0.0)
    _, _, proj, bins = _small(ora, 0, n=120, seed=4)
    W, H = proj["W"], proj["H"]
    rng = np.random.default_rng(6)
    u = (rng.normal(size=(3, H, W)), rng.normal(size=(3, 3, H, W)))
    g = ora.render_adjoint(proj, bins, u, bg=bg)["g2d"]
    base = ora.render(proj, bins, bg=bg)
    vis = np.flatnonzero(proj["tiles_touched"] > 0)
    checked = 0
    for i in vis[:25]:
        for f in range(9):
            val = proj[FIELD[f][0]][i] if FIELD[f][1] is None else proj[FIELD[f][0]][i, FIELD[f][1]]
            h = 1e-7 * max(1.0, abs(val))
            rp = ora.render(_perturbed(proj, i, f, h), bins, bg=bg)
            rm = ora.render(_perturbed(proj, i, f, -h), bins, bg=bg)
            if not (rp["n_acc"] == rm["n_acc"] == base["n_acc"] and
                    np.array_equal(rp["state"][4], base["state"][4]) and
                    np.array_equal(rm["state"][4], base["state"][4])):
                continue
            lp = _dot(u[0], rp["C"]) + _dot(u[1], rp["grads"])
            lm = _dot(u[0], rm["C"]) + _dot(u[1], rm["grads"])
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[i, f]) <= 1e-5 * (abs(fd) + 1e-3 * np.abs(g).max()), (i, f, fd, g[i, f])
            checked += 1
    assert checked >= 150


def test_render_adjoint_color_single_gaussian(ora):
    """One Gaussian over a background: C = c alpha + bg (1 - alpha), so
    dC/dc = alpha, and dC_x/dc = alpha_x = alpha g_x (closed form)."""
    scene = dict(means=np.array([[0.02, -0.01, 3.0]], np.float32),
                 log_scales=np.log(np.array([[0.05, 0.03, 0.04]], np.float32)),
                 quats=np.array([[1.0, 0.0, 0.0, 0.0]], np.float32),
                 opacity_logits=np.array([0.5], np.float32),
                 rgb=np.array([[0.3, 0.6, 0.9]], np.float32))
    W = H = 16
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H, mode=1)
    bins = ora.bin_pairs(proj)
    x, y = 9, 6
    u = np.zeros((1, 12))
    u[0, 0] = 1.0      # dL/dC_r
    u[0, 4] = 1.0      # dL/dCx_g
    g = ora.render_adjoint(proj, bins, u, pixels=np.array([[x, y]]))["g2d"]
    a, b, c = proj["conic"][0]
    dx, dy = x - proj["mean2d"][0, 0], y - proj["mean2d"][0, 1]
    alpha = proj["opacity"][0] * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy))
    gx = -(a * dx + b * dy)
    assert g[0, 6] == pytest.approx(alpha, rel=1e-12)
    assert g[0, 7] == pytest.approx(alpha * gx, rel=1e-12)
    assert g[0, 8] == 0.0


# ---------------------------------------------------------------- projection

def _loss_project(ora, scene, cam, W, H, g2d):
    p = ora.project(scene, cam, W, H, mode=1)
    outs = np.concatenate([p["mean2d"], p["conic"], p["opacity"][:, None], p["rgb"]], 1)
    return _dot(g2d, outs)


@pytest.mark.parametrize("sh", [None, 1, 3])
def test_project_adjoint_fd(ora, sh):
    """Dual-number projection adjoint against FP64 central differences of
    ora.project, for every input of a few Gaussians (rotated camera)."""
    n, W, H = 12, 40, 30
    scene = scenes.random_scene(n=n, seed=21, sh_degree=sh)
    scene = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    cam = scenes.pinhole_camera(W, H, viewmat=scenes.look_at_viewmat((0.4, -0.3, -0.6), (0.0, 0.1, 3.0)))
    rng = np.random.default_rng(8)
    g2d = rng.normal(size=(n, 9))
    got = ora.project_adjoint(scene, cam, W, H, g2d)
    fields = ["means", "log_scales", "quats", "opacity_logits", "sh" if sh is not None else "rgb"]
    for key in fields:
        arr = scene[key]
        flat = arr.reshape(n, -1)
        for i in range(0, n, 3):
            for j in range(flat.shape[1]):
                h = 1e-6 * max(1.0, abs(flat[i, j]))
                sp = dict(scene); sm = dict(scene)
                ap = flat.copy(); am = flat.copy()
                ap[i, j] += h; am[i, j] -= h
                sp[key] = ap.reshape(arr.shape); sm[key] = am.reshape(arr.shape)
                fd = (_loss_project(ora, sp, cam, W, H, g2d) - _loss_project(ora, sm, cam, W, H, g2d)) / (2 * h)
                an = got[key].reshape(n, -1)[i, j]
                assert abs(fd - an) <= 1e-6 * (abs(fd) + 1.0), (key, i, j, fd, an)


def test_project_adjoint_culled_is_zero(ora):
    scene = scenes.random_scene(n=4, seed=2)
    scene["means"] = scene["means"].copy()
    scene["means"][1, 2] = -1.0          # behind the camera
    cam = scenes.pinhole_camera(32, 32)
    got = ora.project_adjoint(scene, cam, 32, 32, np.ones((4, 9)))
    for key in ("means", "log_scales", "quats", "rgb"):
        assert not got[key][1].any()
    assert got["opacity_logits"][1] == 0.0
    assert np.abs(got["means"][0]).sum() > 0


# ---------------------------------------------------------------- end to end

def test_end_to_end_fd_exact(ora):
    """L = <u, upscale(render(project(theta)))> in exact mode: the chained
    adjoints equal central differences through all three forward stages."""
    n, W, H, s = 15, 20, 14, 2
    scene = scenes.random_scene(n=n, seed=33, sh_degree=1, log_scale_mean=-2.0, xy_range=0.6)
    scene = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    cam = scenes.pinhole_camera(W, H)
    bg = (0.1, 0.2, 0.3)
    rng = np.random.default_rng(9)
    u = rng.normal(size=(3, H * s, W * s))

    def loss(sc):
        proj = ora.project(sc, cam, W, H, mode=1)
        r = ora.render(proj, ora.bin_pairs(proj), bg=bg)
        return _dot(u, ora.upscale(r["C"], r["grads"], W * s, H * s))

    proj = ora.project(scene, cam, W, H, mode=1)
    bins = ora.bin_pairs(proj)
    dC, dG = ora.upscale_adjoint(u, W, H)
    g2d = ora.render_adjoint(proj, bins, (dC, dG), bg=bg)["g2d"]
    got = ora.project_adjoint(scene, cam, W, H, g2d)
    for key in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        flat = scene[key].reshape(n, -1)
        for i in (0, 7):
            for j in range(min(flat.shape[1], 5)):
                h = 1e-6 * max(1.0, abs(flat[i, j]))
                ap = flat.copy(); am = flat.copy()
                ap[i, j] += h; am[i, j] -= h
                sp = dict(scene); sm = dict(scene)
                sp[key] = ap.reshape(scene[key].shape); sm[key] = am.reshape(scene[key].shape)
                fd = (loss(sp) - loss(sm)) / (2 * h)
                an = got[key].reshape(n, -1)[i, j]
                assert abs(fd - an) <= 2e-6 * (abs(fd) + 1.0), (key, i, j, fd, an)
