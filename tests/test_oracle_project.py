"""Pins of the oracle's projection (Sec. 4: Sigma' = J W Sigma W^T J^T, EWA
splatting), SH colour and tile binning, against references that do not come
from the oracle: scipy rotations and spherical harmonics, a finite-difference
Jacobian of the pinhole map, numpy eigenvalues, rigid-motion invariance and a
brute-force pixel enumeration of the tile sets."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation
from scipy.special import expit, sph_harm_y

import scenes


def _rotated_camera(W, H):
    vm = scenes.look_at_viewmat(eye=(0.7, -0.4, -0.5), target=(0.05, 0.1, 3.0))
    return scenes.pinhole_camera(W, H, viewmat=vm)


def _pinhole(cam, pc):
    return np.array([cam["fx"] * pc[0] / pc[2] + cam["cx"], cam["fy"] * pc[1] / pc[2] + cam["cy"]])


def _jac_fd(cam, pc, h=1e-6):
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h * max(1.0, abs(pc[k]))
        J[:, k] = (_pinhole(cam, pc + e) - _pinhole(cam, pc - e)) / (2 * e[k])
    return J


def _world_cov(scene, i):
    w, x, y, z = scene["quats"][i].astype(np.float64)
    R = Rotation.from_quat([x, y, z, w]).as_matrix()
    S = np.diag(np.exp(scene["log_scales"][i].astype(np.float64)) ** 2)
    return R @ S @ R.T


def test_mean_and_covariance(ora):
    W, H = 64, 48
    scene = scenes.random_scene(300, seed=1)
    cam = _rotated_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    vm = cam["viewmat"].astype(np.float64)
    K = np.array([[cam["fx"], 0, cam["cx"]], [0, cam["fy"], cam["cy"]], [0, 0, 1.0]])
    lim_x, lim_y = 1.3 * W / (2 * cam["fx"]), 1.3 * H / (2 * cam["fy"])
    checked = 0
    for i in range(300):
        mu = scene["means"][i].astype(np.float64)
        pc = vm[:3, :3] @ mu + vm[:3, 3]
        if pc[2] <= cam["znear"]:
            assert proj["radius"][i] == 0 and proj["tiles_touched"][i] == 0
            continue
        uvw = K @ pc
        np.testing.assert_allclose(proj["mean2d"][i], uvw[:2] / uvw[2], rtol=1e-12)
        if abs(pc[0] / pc[2]) > lim_x or abs(pc[1] / pc[2]) > lim_y:
            continue
        J = _jac_fd(cam, pc)
        Wr = vm[:3, :3]
        cov = J @ Wr @ _world_cov(scene, i) @ Wr.T @ J.T + 0.3 * np.eye(2)
        got = proj["cov2d"][i]
        np.testing.assert_allclose([got[0], got[1], got[2]], [cov[0, 0], cov[0, 1], cov[1, 1]],
                                   rtol=1e-7, atol=1e-9 * np.abs(cov).max())
        Q = np.linalg.inv(cov)
        np.testing.assert_allclose(proj["conic"][i], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-6,
                                   atol=1e-9 * np.abs(Q).max())
        lam = np.linalg.eigvalsh(cov).max()
        assert proj["radius"][i] == math.ceil(3 * math.sqrt(lam))
        assert proj["depth"][i] == pytest.approx(pc[2], rel=1e-14)
        checked += 1
    assert checked > 200
    np.testing.assert_allclose(proj["opacity"], expit(scene["opacity_logits"].astype(np.float64)), rtol=1e-14)


def test_jacobian_clamped_outside_frustum(ora):
    """Outside 1.3 tan(fov/2) the Jacobian is taken at the clamped direction."""
    W, H = 64, 64
    cam = scenes.pinhole_camera(W, H)
    scene = scenes.random_scene(1, seed=0)
    scene["means"][0] = [2.5, -0.3, 2.0]       # x/z = 1.25 > 1.3 * tan(30 deg) = 0.75
    scene["quats"][0] = [1, 0, 0, 0]
    scene["log_scales"][0] = [-2.0, -2.5, -1.5]
    proj = ora.project(scene, cam, W, H)
    lim = 1.3 * W / (2 * cam["fx"])
    pc = scene["means"][0].astype(np.float64)
    pclamp = np.array([lim * pc[2], pc[1], pc[2]])
    J = _jac_fd(cam, pclamp)
    cov = J @ _world_cov(scene, 0) @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(proj["cov2d"][0], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-7)
    np.testing.assert_allclose(proj["mean2d"][0], _pinhole(cam, pc), rtol=1e-13)


def test_rigid_motion_invariance(ora):
    """Moving the world and the camera by the same rigid motion changes nothing
    on screen (pins the use of W inside J W Sigma W^T J^T)."""
    W, H = 48, 40
    scene = scenes.random_scene(200, seed=3)
    cam = _rotated_camera(W, H)
    base = ora.project(scene, cam, W, H)
    G = Rotation.from_rotvec([0.3, -0.7, 0.2])
    tr = np.array([0.4, -1.0, 2.0])
    moved = dict(scene)
    moved["means"] = (G.apply(scene["means"].astype(np.float64)) + tr)
    q = scene["quats"].astype(np.float64)
    r = G * Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], 1))
    qx = r.as_quat()
    moved["quats"] = np.concatenate([qx[:, 3:], qx[:, :3]], 1)
    Gm = np.eye(4)
    Gm[:3, :3] = G.as_matrix()
    Gm[:3, 3] = tr
    cam2 = dict(cam)
    cam2["viewmat"] = cam["viewmat"].astype(np.float64) @ np.linalg.inv(Gm)
    got = ora.project(moved, cam2, W, H)
    vis = base["tiles_touched"] > 0
    np.testing.assert_allclose(got["mean2d"][vis], base["mean2d"][vis], rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(got["cov2d"][vis], base["cov2d"][vis], rtol=1e-9, atol=1e-12)


def _real_sh_scipy(deg, dirs):
    d = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    out = np.zeros((len(d), (deg + 1) ** 2))
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)      # complex, Condon-Shortley phase
            if m == 0:
                v = Y.real
            elif m > 0:
                v = math.sqrt(2) * Y.real
            else:
                v = math.sqrt(2) * Y.imag
            out[:, l * l + l + m] = v
    return out


def test_sh_basis_against_scipy(ora):
    rng = np.random.default_rng(0)
    dirs = rng.normal(0, 1, (200, 3))
    dirs[0] = [0, 0, 1]
    dirs[1] = [0, 0, -1]
    got = ora.sh_basis(3, dirs)
    want = _real_sh_scipy(3, dirs)
    np.testing.assert_allclose(got, want, atol=1e-13)
    # l = 1 is (-y, z, -x) times sqrt(3 / (4 pi)) in this convention
    d = dirs[2] / np.linalg.norm(dirs[2])
    c1 = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(got[2, 1:4], [-c1 * d[1], c1 * d[2], -c1 * d[0]], atol=1e-14)


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_colour_from_sh(ora, deg):
    W, H = 32, 32
    scene = scenes.random_scene(100, seed=deg, sh_degree=deg)
    cam = _rotated_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    campos = np.linalg.inv(cam["viewmat"].astype(np.float64))[:3, 3]
    dirs = scene["means"].astype(np.float64) - campos
    Y = _real_sh_scipy(deg, dirs)
    want = np.maximum(0, np.einsum("nk,nkc->nc", Y, scene["sh"].astype(np.float64)) + 0.5)
    vis = proj["radius"] > 0
    # the oracle takes the camera centre as -R^T t; the float32 view matrix is
    # orthonormal only to ~1e-8, hence the absolute tolerance
    np.testing.assert_allclose(proj["rgb"][vis], want[vis], rtol=0, atol=2e-8)


@pytest.mark.parametrize("W,H,seed", [(50, 37, 0), (16, 16, 1), (33, 70, 2)])
def test_binning_brute_force(ora, W, H, seed):
    """The pair list is exactly the set of (tile, Gaussian) with a pixel centre of
    the tile inside the Gaussian's 3-sigma square cut to the bounding box of its
    alpha >= 1/255 ellipse, ordered by tile, FP32 depth, id; ranges delimit each
    tile's run."""
    scene = scenes.random_scene(40, seed=seed, xy_range=1.6)
    cam = _rotated_camera(W, H)
    tile = 16
    proj = ora.project(scene, cam, W, H, tile=tile)
    bins = ora.bin_pairs(proj)
    tx = (W + tile - 1) // tile
    want = []
    for i in range(40):
        r = int(proj["radius"][i])
        if r == 0:
            continue
        mx, my = proj["mean2d"][i]
        L = math.log(255 * proj["opacity"][i])
        if L <= 0:
            assert proj["tiles_touched"][i] == 0
            continue
        # bounding box of the ellipse {d : d^T cov^-1 d <= 2L}, measured on its
        # boundary traced from the eigen-decomposition (sampling error < 1e-6)
        c = proj["cov2d"][i]
        cov = np.array([[c[0], c[1]], [c[1], c[2]]])
        lam, vec = np.linalg.eigh(cov)
        th = np.linspace(0, 2 * np.pi, 20001)
        pts = vec @ (np.sqrt(2 * L * lam)[:, None] * np.stack([np.cos(th), np.sin(th)]))
        hx = min(r, np.abs(pts[0]).max())
        hy = min(r, np.abs(pts[1]).max())
        tiles = set()
        for py in range(H):
            if abs(py - my) > hy:
                continue
            for px in range(W):
                if abs(px - mx) <= hx:
                    tiles.add((py // tile) * tx + px // tile)
        if proj["borderline"][i]:
            continue
        assert len(tiles) == proj["tiles_touched"][i]
        d32 = np.float32(proj["depth"][i]).view(np.uint32)
        want += [(t, int(d32), i) for t in tiles]
    keep = set(np.nonzero(proj["borderline"] == 0)[0].tolist())
    want.sort()
    got = [(int(k >> np.uint64(32)), int(k & np.uint64(0xFFFFFFFF)), int(v))
           for k, v in zip(bins["keys"], bins["vals"]) if int(v) in keep]
    assert got == want
    ranges = bins["ranges"]
    allp = [(int(k >> np.uint64(32)), int(v)) for k, v in zip(bins["keys"], bins["vals"])]
    for t in range(ranges.shape[0]):
        s, e = ranges[t]
        run = [g for g in allp if g[0] == t]
        assert e - s == len(run)
        if run:
            assert allp[s:e] == run


@pytest.mark.parametrize("seed", [0, 1])
def test_tight_tile_sets_keep_the_image(ora, seed):
    """Binning each Gaussian only into the tiles of its alpha >= 1/255 box drops
    only pairs the cut-off rejects: the 3DGS-mode image (colour, derivatives,
    state) is bit-identical to binning every Gaussian into every tile."""
    W, H = 48, 40
    scene = scenes.random_scene(400, seed=seed, sh_degree=1)
    cam = _rotated_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    full = dict(proj)
    vis = proj["radius"] > 0
    full["rect"] = np.where(vis[:, None], np.array([0, 0, full["tiles_x"] - 1, full["tiles_y"] - 1]),
                            np.array([0, 0, -1, -1])).astype(np.int32)
    full["tiles_touched"] = np.where(vis, full["tiles_x"] * full["tiles_y"], 0).astype(np.int64)
    a = ora.render(proj, ora.bin_pairs(proj))
    b = ora.render(full, ora.bin_pairs(full))
    assert ora.bin_pairs(proj)["P"] < 0.5 * ora.bin_pairs(full)["P"]
    np.testing.assert_array_equal(a["C"], b["C"])
    np.testing.assert_array_equal(a["grads"], b["grads"])
    np.testing.assert_array_equal(a["state"][:4], b["state"][:4])


def _square_rects(proj):
    """The 3DGS renderer's tile sets: the tiles holding a pixel centre (i, j)
    with |i - mean_x| <= r and |j - mean_y| <= r, r = the radius
    ceil(3 sqrt(lambda_max)), clipped to the image."""
    W, H, tile = proj["W"], proj["H"], proj["tile"]
    r = np.asarray(proj["radius"], np.float64)
    mx, my = np.asarray(proj["mean2d"], np.float64).T
    x0, x1 = np.ceil(mx - r), np.floor(mx + r)
    y0, y1 = np.ceil(my - r), np.floor(my + r)
    ok = (r > 0) & (x1 >= 0) & (x0 <= W - 1) & (y1 >= 0) & (y0 <= H - 1) & (x0 <= x1) & (y0 <= y1)
    rect = np.stack([np.clip(x0, 0, W - 1) // tile, np.clip(y0, 0, H - 1) // tile,
                     np.clip(x1, 0, W - 1) // tile, np.clip(y1, 0, H - 1) // tile], 1).astype(np.int32)
    rect[~ok] = np.array([0, 0, -1, -1], np.int32)
    touched = np.where(ok, (rect[:, 2] - rect[:, 0] + 1) * (rect[:, 3] - rect[:, 1] + 1), 0).astype(np.int64)
    return rect, touched


@pytest.mark.slow
def test_tight_tile_sets_keep_the_image_dense_opaque(ora):
    """At the benchmark scene's density (about 3 Gaussians per pixel: 18,000
    over 96 x 64) with mostly opaque Gaussians (opacity logits N(1, 1), sigma
    above 0.35 for 84 % of them).  For such Gaussians the alpha >= 1/255
    ellipse reaches past the 3-sigma square, so the square (the 3DGS renderer's
    own truncation, which every-tile binning would not apply) is the
    reference: cutting it to the alpha >= 1/255 box drops only pairs the
    cut-off rejects, and the image is bit-identical to the square's."""
    W, H = 96, 64
    scene = scenes.random_scene(18000, seed=7, sh_degree=1, xy_range=1.0, log_scale_mean=-3.3)
    scene["opacity_logits"] = np.random.default_rng(7).normal(1.0, 1.0, 18000).astype(np.float32)
    sig = 1.0 / (1.0 + np.exp(-scene["opacity_logits"].astype(np.float64)))
    assert np.mean(sig > 0.35) > 0.8
    cam = _rotated_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    square = dict(proj)
    square["rect"], square["tiles_touched"] = _square_rects(proj)
    tight = ora.bin_pairs(proj)
    full = ora.bin_pairs(square)
    assert tight["P"] < 0.9 * full["P"]          # the cut removes pairs inside the squares (15 % here)
    a = ora.render(proj, tight)
    b = ora.render(square, full)
    np.testing.assert_array_equal(a["C"], b["C"])
    np.testing.assert_array_equal(a["grads"], b["grads"])
    np.testing.assert_array_equal(a["state"][:4], b["state"][:4])
    # and the square does truncate here: binning every Gaussian into every
    # tile changes the image (alpha >= 1/255 beyond 3 sigma)
    every = dict(proj)
    vis = proj["radius"] > 0
    every["rect"] = np.where(vis[:, None], np.array([0, 0, every["tiles_x"] - 1, every["tiles_y"] - 1]),
                             np.array([0, 0, -1, -1])).astype(np.int32)
    every["tiles_touched"] = np.where(vis, every["tiles_x"] * every["tiles_y"], 0).astype(np.int64)
    c = ora.render(every, ora.bin_pairs(every))
    assert not np.array_equal(a["C"], c["C"])


def test_borderline_flags_are_rare(ora):
    W, H = 64, 64
    scene = scenes.random_scene(1000, seed=0)
    proj = ora.project(scene, scenes.pinhole_camera(W, H), W, H)
    assert proj["borderline"].sum() <= 2
