"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs, at sizes that span several tiles, ragged image edges and
several radix-sort tiles (4096 keys), plus the degenerate cases."""
import numpy as np
import pytest

import scenes
from helpers import (TOL_UP, borderline_tile_mask, compare_pixels, compare_render, gpu_rows, pairs_without)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import torch
    import paper_2503_14171_gb300 as gs
    assert torch.cuda.is_available()
    return gs


def _rotated(W, H, eye=(0.7, -0.4, -0.5), target=(0.05, 0.1, 3.0)):
    return scenes.pinhole_camera(W, H, viewmat=scenes.look_at_viewmat(eye, target))


def _translated(W, H, t=(0.1, -0.05, 0.3)):
    vm = np.eye(4, dtype=np.float32)
    vm[:3, 3] = t
    return scenes.pinhole_camera(W, H, viewmat=vm)


CASES = [
    # name, scene kwargs, camera, W, H
    ("cfg1_64", dict(n=1000, seed=0), "ident", 64, 64),
    ("ragged_sh3", dict(n=3000, seed=5, sh_degree=3), "rot", 77, 45),
    ("sh1_translated", dict(n=2000, seed=7, sh_degree=1), "trans", 50, 70),
    ("dense_many_tiles", dict(n=30000, seed=3, xy_range=1.3, log_scale_mean=-3.4), "ident", 200, 136),
]


def _cam(kind, W, H):
    return {"ident": scenes.pinhole_camera, "rot": _rotated, "trans": _translated}[kind](W, H)


@pytest.mark.parametrize("name,kw,camkind,W,H", CASES)
def test_projection(gs, ora, name, kw, camkind, W, H):
    scene = scenes.random_scene(**kw)
    cam = _cam(camkind, W, H)
    ref = ora.project(scene, cam, W, H)
    with gs.Context() as ctx:
        ctx.project(gs.DeviceScene(scene), cam, W, H)
        got = {k: v.cpu().numpy() for k, v in ctx.read_projected().items()}
    vis = ref["radius"] > 0
    ok = vis & (ref["borderline"] == 0)
    assert np.array_equal(got["radius"] > 0, vis)
    assert np.array_equal(got["radius"][ok], ref["radius"][ok])
    assert np.array_equal(got["tiles_touched"][ok], ref["tiles_touched"][ok])
    m = ref["mean2d"][vis]
    np.testing.assert_allclose(got["mean2d"][vis], m, rtol=0, atol=2e-6 * (np.abs(m).max() + 100))
    cscale = np.abs(ref["conic"][vis]).max(axis=1, keepdims=True)
    assert np.all(np.abs(got["conic"][vis] - ref["conic"][vis]) <= 2e-5 * cscale)
    np.testing.assert_allclose(got["rgb"][vis], ref["rgb"][vis], rtol=0, atol=2e-6)
    np.testing.assert_allclose(got["opacity"][vis], ref["opacity"][vis], rtol=2e-6)
    np.testing.assert_allclose(got["depth"][vis], ref["depth"][vis], rtol=2e-7)


@pytest.mark.parametrize("name,kw,camkind,W,H", [c for c in CASES if c[2] != "rot"])
def test_bins_bit_exact(gs, ora, name, kw, camkind, W, H):
    """Keys (tile << 32 | FP32 depth bits), ids and per-tile ranges equal the
    oracle's bit for bit (identity-rotation cameras, where the FP32 depth is
    exact); pairs of borderline Gaussians are compared as sets."""
    scene = scenes.random_scene(**kw)
    cam = _cam(camkind, W, H)
    proj = ora.project(scene, cam, W, H)
    ref = ora.bin_pairs(proj)
    with gs.Context() as ctx:
        ctx.project(gs.DeviceScene(scene), cam, W, H)
        keys, vals, ranges = (t.cpu().numpy() for t in ctx.read_bins())
    keys = keys.view(np.uint64)
    vals = vals.view(np.uint32)
    drop = np.nonzero(proj["borderline"])[0].astype(np.uint32)
    gk, gv = pairs_without(keys, vals, drop)
    rk, rv = pairs_without(ref["keys"], ref["vals"], drop)
    assert np.array_equal(gk, rk)
    assert np.array_equal(gv, rv)
    if len(drop) == 0:
        assert np.array_equal(ranges.view(np.uint32), ref["ranges"])
    # ranges are consistent with the GPU's own list either way
    t = (keys >> np.uint64(32)).astype(np.int64)
    for tile in np.unique(t)[:50]:
        s, e = ranges.view(np.uint32)[tile]
        assert np.all(t[s:e] == tile)


@pytest.mark.parametrize("W,H,side", [(256, 256, 1), (512, 288, 2), (1024, 576, 4), (1040, 600, 4)])
def test_bins_bit_exact_every_super_side(gs, ora, W, H, side):
    """The per-frame super-tile side (1, 2 or 4 tiles: the smallest with at
    most 256 super-tiles) at sizes that pick each: the per-tile lists equal
    the oracle's bit for bit, the super-tile pair count is the one that side
    gives, and sampled pixels of the derivative render match the oracle."""
    scene = scenes.random_scene(n=30000, seed=27, sh_degree=1, xy_range=1.2, log_scale_mean=-3.8)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    ref = ora.bin_pairs(proj)
    tx, ty = (W + 15) // 16, (H + 15) // 16
    assert side == next(k for k in (1, 2, 4) if ((tx + k - 1) // k) * ((ty + k - 1) // k) <= 256 or k == 4)
    # super-tile pairs the side gives, from the oracle's rects
    rc = np.asarray(proj["rect"], np.int64)
    live = rc[:, 2] >= rc[:, 0]
    want_ps = int(np.sum(((rc[live, 2] // side) - (rc[live, 0] // side) + 1) *
                         ((rc[live, 3] // side) - (rc[live, 1] // side) + 1)))
    rng = np.random.default_rng(W)
    pix = np.stack([rng.integers(0, W, 600), rng.integers(0, H, 600)], 1)
    with gs.Context() as ctx:
        dev = gs.DeviceScene(scene)
        C, G = ctx.render_with_grads(dev, cam, W, H)
        keys, vals, _ = (t.cpu().numpy() for t in ctx.read_bins())
        ps = ctx.super_pair_count()
        rows = gpu_rows(C, G, pix)
    drop = np.nonzero(proj["borderline"])[0].astype(np.uint32)
    gk, gv = pairs_without(keys.view(np.uint64), vals.view(np.uint32), drop)
    rk, rv = pairs_without(ref["keys"], ref["vals"], drop)
    assert len(rk) > 10000
    assert np.array_equal(gk, rk) and np.array_equal(gv, rv)
    if len(drop) == 0:
        assert ps == want_ps
    out = ora.render(proj, ref, pixels=pix, variants=True)
    excl = borderline_tile_mask(proj)[pix[:, 1], pix[:, 0]]
    fail, checked, _ = compare_pixels(rows, out, exclude=excl)
    assert fail == 0 and checked > 0.9 * len(pix), (fail, checked)


def _wide_depth_scene(n=6000, seed=21, z=(0.02, 3000.0)):
    """Depths log-uniform over a ratio of 150,000 (beyond the 2^27 FP32 steps
    that three 9-bit radix passes cover), positions and scales in proportion
    to depth so that every depth is on screen at a similar pixel size."""
    scene = scenes.random_scene(n=n, seed=seed)
    rng = np.random.default_rng(seed + 1)
    d = np.exp(rng.uniform(np.log(z[0]), np.log(z[1]), n))
    scene["means"][:, 2] = d
    scene["means"][:, :2] *= (0.5 * d)[:, None]
    scene["log_scales"] += np.log(0.6 * d).astype(np.float32)[:, None]
    return scene


@pytest.mark.parametrize("z", [(0.02, 3000.0), (0.5, 8.0)])
def test_bins_bit_exact_over_depth_ranges(gs, ora, z):
    """The depth sort biases the FP32 depth bits by the smallest visible one and
    takes three 9-bit passes when the visible keys' span plus the Gaussian
    count fits 27 bits, four otherwise: both cases against the oracle's bins,
    bit for bit."""
    W, H = 96, 64
    scene = _wide_depth_scene(z=z)
    cam = scenes.pinhole_camera(W, H, znear=0.01)
    proj = ora.project(scene, cam, W, H)
    vis = proj["tiles_touched"] > 0
    bits = proj["depth"][vis].astype(np.float32).view(np.uint32).astype(np.int64)
    span = int(bits.max() - bits.min())
    n = len(proj["depth"])
    assert (span + n >= (1 << 27)) == (z[1] / z[0] > 65536)   # the case this parameter is meant to hit
    ref = ora.bin_pairs(proj)
    with gs.Context() as ctx:
        ctx.project(gs.DeviceScene(scene), cam, W, H)
        keys, vals, ranges = (t.cpu().numpy() for t in ctx.read_bins())
    drop = np.nonzero(proj["borderline"])[0].astype(np.uint32)
    gk, gv = pairs_without(keys.view(np.uint64), vals.view(np.uint32), drop)
    rk, rv = pairs_without(ref["keys"], ref["vals"], drop)
    assert len(rk) > 1000
    assert np.array_equal(gk, rk)
    assert np.array_equal(gv, rv)


@pytest.mark.parametrize("name,kw,camkind,W,H", CASES)
@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.2, 0.5, 0.9)])
def test_render_with_grads(gs, ora, name, kw, camkind, W, H, bg):
    scene = scenes.random_scene(**kw)
    cam = _cam(camkind, W, H)
    proj = ora.project(scene, cam, W, H)
    bins = ora.bin_pairs(proj)
    ref = ora.render(proj, bins, bg=bg, variants=True)
    with gs.Context(bg=bg) as ctx:
        C, G = ctx.render_with_grads(gs.DeviceScene(scene), cam, W, H)
        ctx.synchronize()
        C, G = C.cpu().numpy(), G.cpu().numpy()
    fail, checked, excl, worst = compare_render(C, G, ref, exclude=borderline_tile_mask(proj))
    assert fail == 0, f"{fail} of {checked} pixels outside tolerance (worst {worst:.2f}x tol)"
    assert checked > 0.9 * W * H, (checked, excl)


@pytest.mark.parametrize("name,kw,camkind,W,H", CASES[:2])
def test_plain_render(gs, ora, name, kw, camkind, W, H):
    scene = scenes.random_scene(**kw)
    cam = _cam(camkind, W, H)
    proj = ora.project(scene, cam, W, H)
    bins = ora.bin_pairs(proj)
    ref = ora.render(proj, bins, variants=True)
    with gs.Context() as ctx:
        C = ctx.render(gs.DeviceScene(scene), cam, W, H).cpu().numpy()
    fail, checked, excl, _ = compare_render(C, None, ref, exclude=borderline_tile_mask(proj))
    assert fail == 0 and checked > 0.9 * W * H


def test_state_and_count(gs, ora):
    W, H = 64, 48
    scene = scenes.random_scene(1500, seed=12)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    bins = ora.bin_pairs(proj)
    ref = ora.render(proj, bins, variants=True)
    with gs.Context() as ctx:
        ctx.render_with_grads(gs.DeviceScene(scene), cam, W, H)
        state, count = (t.cpu().numpy() for t in ctx.read_state())
    clean = (ref["nvar"] == 1) & ~borderline_tile_mask(proj)
    # T_N = 1 - A_N and its derivatives are -A_N's
    np.testing.assert_allclose(state[0][clean], 1 - ref["state"][0][clean], atol=2e-4)
    for k in (1, 2, 3):
        r = ref["state"][k]
        tol = 1e-3 * np.maximum(np.abs(r), np.sqrt(np.mean(r ** 2)))
        assert np.all(np.abs(state[k] + r)[clean] <= tol[clean])
    assert np.array_equal(count[clean], ref["state"][4][clean].astype(np.int32))


def test_exact_mode(gs, ora):
    """No cut-offs, every Gaussian in every tile: a smooth image, all pixels compared."""
    W, H = 45, 38
    scene = scenes.random_scene(60, seed=21, xy_range=0.7)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H, mode=ora.MODE_EXACT)
    bins = ora.bin_pairs(proj)
    ref = ora.render(proj, bins, variants=True)
    assert np.all(ref["nvar"] == 1)
    with gs.Context(mode="exact") as ctx:
        C, G = ctx.render_with_grads(gs.DeviceScene(scene), cam, W, H)
        C, G = C.cpu().numpy(), G.cpu().numpy()
    fail, checked, excl, worst = compare_render(C, G, ref)
    assert fail == 0 and excl == 0, worst


@pytest.mark.parametrize("W,H", [(1, 1), (17, 1), (1, 33), (16, 16), (31, 17)])
def test_tiny_and_ragged_images(gs, ora, W, H):
    scene = scenes.random_scene(400, seed=W * 100 + H, xy_range=0.5)
    cam = scenes.pinhole_camera(max(W, 2), max(H, 2))
    cam["cx"], cam["cy"] = (W - 1) / 2, (H - 1) / 2
    proj = ora.project(scene, cam, W, H)
    bins = ora.bin_pairs(proj)
    ref = ora.render(proj, bins, variants=True)
    with gs.Context() as ctx:
        C, G = ctx.render_with_grads(gs.DeviceScene(scene), cam, W, H)
        C, G = C.cpu().numpy(), G.cpu().numpy()
    fail, checked, excl, worst = compare_render(C, G, ref, exclude=borderline_tile_mask(proj))
    assert fail == 0, worst


def test_empty_and_culled(gs):
    """No Gaussians, or all behind the near plane: background everywhere, zero derivatives."""
    W, H = 40, 24
    bg = (0.1, 0.2, 0.3)
    cam = scenes.pinhole_camera(W, H)
    empty = scenes.random_scene(0, seed=0)
    behind = scenes.random_scene(500, seed=1)
    behind["means"][:, 2] = -behind["means"][:, 2]
    with gs.Context(bg=bg) as ctx:
        for sc in (empty, behind):
            C, G = ctx.render_with_grads(gs.DeviceScene(sc), cam, W, H)
            assert ctx.pair_count() == 0
            C, G = C.cpu().numpy(), G.cpu().numpy()
            for ch in range(3):
                assert np.all(C[ch] == np.float32(bg[ch]))
            assert np.all(G == 0)


def test_capacity_limit_reports_error(gs):
    W, H = 64, 64
    scene = scenes.random_scene(1000, seed=0)
    cam = scenes.pinhole_camera(W, H)
    with gs.Context(max_pairs=100) as ctx:
        with pytest.raises(gs.GSError) as ei:
            ctx.render_with_grads(gs.DeviceScene(scene), cam, W, H)
        assert ei.value.status == gs.GS_ERR_CAPACITY
        # the context stays usable after the error
        ctx.set_options(max_pairs=0)
        ctx.render_with_grads(gs.DeviceScene(scene), cam, W, H)
        ctx.synchronize()


@pytest.mark.parametrize("W,H,s", [(64, 64, 2), (23, 17, 3), (40, 9, 4), (5, 4, 8), (12, 7, 1), (3, 2, 16),
                                   (97, 61, 5)])
def test_upscale_matches_oracle(gs, ora, W, H, s):
    import torch
    rng = np.random.default_rng(W * 31 + H * 7 + s)
    C = rng.uniform(0, 1, (3, H, W)).astype(np.float32)
    G = rng.normal(0, 0.3, (3, 3, H, W)).astype(np.float32)
    with gs.Context() as ctx:
        out = ctx.upscale(torch.from_numpy(C).cuda(), torch.from_numpy(G).cuda(), s).cpu().numpy()
    ref = ora.upscale(C.astype(np.float64), G.astype(np.float64), s * W, s * H)
    scale = 1 + max(np.abs(C).max(), np.abs(G).max())
    assert np.abs(out - ref).max() <= TOL_UP * scale


def test_upscale_of_rendered_image(gs, ora):
    """Render (GPU) -> upscale (GPU) equals the oracle's upscale of the GPU render,
    and the oracle's render -> upscale within the propagated render tolerance."""
    import torch  # noqa: F401
    W, H, s = 64, 64, 2
    scene = scenes.random_scene(1000, seed=0)
    cam = scenes.pinhole_camera(W, H)
    with gs.Context() as ctx:
        C, G = ctx.render_with_grads(gs.DeviceScene(scene), cam, W, H)
        up = ctx.upscale(C, G, s).cpu().numpy()
        Cn, Gn = C.cpu().numpy().astype(np.float64), G.cpu().numpy().astype(np.float64)
    ref = ora.upscale(Cn, Gn, s * W, s * H)
    assert np.abs(up - ref).max() <= TOL_UP * (1 + np.abs(Gn).max())


@pytest.mark.parametrize("W,H,factor", [(1, 5, 2), (5, 1, 2), (8, 8, 0), (8, 8, 17)])
def test_upscale_rejects_bad_arguments(gs, W, H, factor):
    import torch
    with gs.Context() as ctx:
        C = torch.zeros(3, H, W, device="cuda")
        G = torch.zeros(3, 3, H, W, device="cuda")
        out = torch.zeros(3, max(1, H * max(factor, 1)), max(1, W * max(factor, 1)), device="cuda")
        with pytest.raises(gs.GSError) as ei:
            gs.gs_upscale(ctx.h, C.data_ptr(), G.data_ptr(), W, H, factor, out.data_ptr())
        assert ei.value.status == gs.GS_ERR_INVALID_ARG


def test_repeated_calls_are_deterministic(gs):
    W, H = 96, 64
    scene = scenes.random_scene(5000, seed=8, sh_degree=2)
    cam = _rotated(W, H)
    dev = gs.DeviceScene(scene)
    with gs.Context() as ctx:
        C1, G1 = (t.clone() for t in ctx.render_with_grads(dev, cam, W, H))
        C2, G2 = ctx.render_with_grads(dev, cam, W, H)
        assert bool((C1 == C2).all()) and bool((G1 == G2).all())


def test_blend_work_counts_match_oracle(gs, ora):
    """The counting variant of the blend visits exactly the oracle's (pixel,
    Gaussian) pairs: every list entry before a pixel stops, and the blended ones."""
    W, H = 64, 64
    scene = scenes.random_scene(1000, seed=0)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    ref = ora.render(proj, ora.bin_pairs(proj))
    with gs.Context() as ctx:
        ctx.project(gs.DeviceScene(scene), cam, W, H)
        n_eval, n_acc = ctx.blend_stats()
    assert abs(n_eval - ref["n_eval"]) <= 2e-3 * ref["n_eval"]
    assert abs(n_acc - ref["n_acc"]) <= 2e-3 * ref["n_acc"]


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_projection_of_unaligned_sh(gs, shift):
    """SH coefficients starting off a 16-byte boundary (a view into a larger
    buffer) take the projection's scalar staging path; the projected records,
    bins and image equal those of the aligned copy bit for bit."""
    import torch
    scene = scenes.random_scene(n=3000, seed=41, sh_degree=3, xy_range=1.2)
    W, H = 80, 56
    cam = scenes.pinhole_camera(W, H)
    aligned = gs.DeviceScene(scene)
    sh = np.ascontiguousarray(scene["sh"], np.float32).reshape(-1)
    buf = torch.zeros(sh.size + 4, dtype=torch.float32, device="cuda")
    buf[shift:shift + sh.size] = torch.as_tensor(sh).cuda()
    tensors = dict(aligned.t)
    tensors["sh"] = buf[shift:shift + sh.size].view(scene["sh"].shape)
    assert tensors["sh"].data_ptr() % 16 != 0
    shifted = gs.DeviceScene(scene, tensors=tensors)
    res = []
    for dev in (aligned, shifted):
        with gs.Context() as ctx:
            C, G = ctx.render_with_grads(dev, cam, W, H)
            pr = {k: v.cpu().numpy() for k, v in ctx.read_projected().items()}
            res.append((C.cpu().numpy(), G.cpu().numpy(), pr))
    (C0, G0, p0), (C1, G1, p1) = res
    assert np.array_equal(C0, C1) and np.array_equal(G0, G1)
    for k in p0:
        assert np.array_equal(p0[k], p1[k]), k


def test_exact_mode_escaped_pair_counts(gs, ora):
    """A frame of 2050 super-tiles in exact mode: every Gaussian touches every
    super-tile, so its pair count (2050) exceeds the 11 bits that ride with
    its id through the depth sort and is looked up.  The bins equal the
    oracle's bit for bit, and sampled pixels match."""
    W, H = 3200, 2624
    scene = scenes.random_scene(40, seed=24, xy_range=0.6)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H, mode=ora.MODE_EXACT)
    vis = proj["tiles_touched"] > 0
    assert vis.sum() > 20
    ref_bins = ora.bin_pairs(proj)
    rng = np.random.default_rng(3)
    pix = np.stack([rng.integers(0, W, 800), rng.integers(0, H, 800)], 1)
    ref = ora.render(proj, ref_bins, pixels=pix, variants=True)
    with gs.Context(mode="exact") as ctx:
        dev = gs.DeviceScene(scene)
        C, G = ctx.render_with_grads(dev, cam, W, H)
        keys, vals, _ = (t.cpu().numpy() for t in ctx.read_bins())
        rows = gpu_rows(C, G, pix)
    assert np.array_equal(keys.view(np.uint64), ref_bins["keys"])
    assert np.array_equal(vals.view(np.uint32), ref_bins["vals"])
    fail, checked, excluded = compare_pixels(rows, ref)
    assert fail == 0 and checked == len(pix), (fail, checked, excluded)


def test_invalid_gaussians_are_culled(gs):
    """Gaussians with a NaN mean, NaN log-scales, a NaN opacity logit or a zero
    quaternion are culled: the render (with derivatives) equals, bit for bit,
    the render of the scene without them, and the pair count is theirs less."""
    scene = scenes.random_scene(n=2000, seed=26, sh_degree=2, xy_range=1.1)
    bad = scenes.random_scene(n=2000, seed=26, sh_degree=2, xy_range=1.1)
    bad["means"][0:10, 0] = np.nan
    bad["log_scales"][10:20, 1] = np.nan
    bad["opacity_logits"][20:30] = np.nan
    bad["quats"][30:40] = 0.0
    keep = np.ones(2000, bool)
    keep[:40] = False
    good = {k: (v[keep] if isinstance(v, np.ndarray) and v.shape[:1] == (2000,) else v) for k, v in scene.items()}
    W, H = 96, 80
    cam = scenes.pinhole_camera(W, H)
    out = []
    for sc in (bad, good):
        with gs.Context() as ctx:
            C, G = ctx.render_with_grads(gs.DeviceScene(sc), cam, W, H)
            out.append((C.cpu().numpy(), G.cpu().numpy(), ctx.pair_count()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]
