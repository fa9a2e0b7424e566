"""GPU parity of the reverse mode (supplement "Backward Pass"): each adjoint
kernel, through the C ABI, against the FP64 oracle's adjoint on the same
upstream gradient.

Both variants of the blend adjoint are checked: the inversion trick from the
forward's stored final state, and the recompute variant (the tile's forward
walk re-run, the exact state checkpointed at each round of candidates).

Tolerances: gradients are sums of many FP32 terms (per pixel a back-to-front
sweep with the state recovered by dividing by 1 - alpha, then atomics across
pixels), so a Gaussian's gradient is compared as
    |gpu - ref| <= TOL_REL |ref| + TOL_ABS rms(ref column over Gaussians),
TOL = 5e-4: the largest error seen on these cases is 5.6e-5 of |ref| + rms
(the dense case), i.e. a margin of about 9x.
In 3DGS mode the upstream gradient is zeroed on the pixels the forward parity
tests exclude (near-threshold decisions, tiles of rect-borderline Gaussians),
so both sides sum over pixels whose blend decisions agree."""
import numpy as np
import pytest

import scenes
from helpers import borderline_tile_mask

pytestmark = pytest.mark.gpu

TOL_REL = 5e-4
TOL_ABS = 5e-4
TOL_UP_BWD = 2e-6


@pytest.fixture(scope="module")
def gs():
    import torch
    import paper_2503_14171_gb300 as gs
    assert torch.cuda.is_available()
    return gs


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()


def _cmp_cols(got, ref, tol_rel=TOL_REL, tol_abs=TOL_ABS):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    rms = np.sqrt(np.mean(ref ** 2, axis=0, keepdims=True)) + 1e-30
    tol = tol_rel * np.abs(ref) + tol_abs * rms
    bad = np.abs(got - ref) > tol
    worst = float(np.max(np.abs(got - ref) / tol)) if got.size else 0.0
    return int(bad.sum()), worst


# ---------------------------------------------------------------- upscale

@pytest.mark.parametrize("W,H,s", [(64, 48, 2), (77, 45, 3), (33, 17, 4), (2, 2, 5), (40, 30, 1), (19, 23, 16)])
def test_upscale_backward(gs, ora, W, H, s):
    rng = np.random.default_rng(W + 7 * s)
    dout = rng.normal(size=(3, H * s, W * s)).astype(np.float32)
    want_C, want_G = ora.upscale_adjoint(dout.astype(np.float64), W, H)
    with gs.Context() as ctx:
        dC, dG = ctx.upscale_backward(_t(dout), W, H, s)
        dC, dG = dC.cpu().numpy(), dG.cpu().numpy()
    scale = 1.0 + np.abs(dout).max() * (2 * s + 2) ** 2
    assert np.abs(dC - want_C).max() <= TOL_UP_BWD * scale
    assert np.abs(dG - want_G).max() <= TOL_UP_BWD * scale


# ---------------------------------------------------------------- blend

CASES = [
    # name, scene kwargs, W, H, mode, bg
    ("cfg1_64", dict(n=1000, seed=0), 64, 64, "3dgs", (0.0, 0.0, 0.0)),
    ("ragged_sh3_bg", dict(n=3000, seed=5, sh_degree=3), 77, 45, "3dgs", (0.3, 0.1, 0.7)),
    ("dense", dict(n=20000, seed=3, xy_range=1.3, log_scale_mean=-3.4), 120, 96, "3dgs", (0.0, 0.0, 0.0)),
    ("exact", dict(n=400, seed=9, log_scale_mean=-2.5), 48, 40, "exact", (0.2, 0.2, 0.2)),
]


VARIANTS = ["inversion", "recompute"]


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("name,kw,W,H,mode,bg", CASES)
def test_render_backward(gs, ora, name, kw, W, H, mode, bg, variant):
    scene = scenes.random_scene(**kw)
    cam = scenes.pinhole_camera(W, H)
    m = 0 if mode == "3dgs" else 1
    proj = ora.project(scene, cam, W, H, mode=m)
    bins = ora.bin_pairs(proj)
    rng = np.random.default_rng(3)
    uC = rng.normal(size=(3, H, W))
    uG = rng.normal(size=(3, 3, H, W))
    if mode == "3dgs":
        ref = ora.render(proj, bins, bg=bg, variants=True)
        keep = (ref["nvar"] == 1) & ~borderline_tile_mask(proj)
        assert keep.mean() > 0.9
        uC = uC * keep
        uG = uG * keep
    want = ora.render_adjoint(proj, bins, (uC, uG), bg=bg)["g2d"]
    with gs.Context(mode=mode, bg=bg, bwd_recompute=variant == "recompute") as ctx:
        ctx.render_with_grads(gs.DeviceScene(scene), cam, W, H)
        got = ctx.render_backward(_t(uC), _t(uG)).cpu().numpy()
        ctx.synchronize()
    assert got.shape == want.shape
    assert np.all(np.isfinite(got))
    bad, worst = _cmp_cols(got, want)
    assert bad == 0, (bad, worst)


def test_render_backward_colour_only(gs, ora):
    """dL_dgrads = NULL: the upstream gradient of the colour image alone."""
    W, H = 64, 48
    scene = scenes.random_scene(n=1500, seed=12)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    bins = ora.bin_pairs(proj)
    ref = ora.render(proj, bins, variants=True)
    keep = (ref["nvar"] == 1) & ~borderline_tile_mask(proj)
    uC = np.random.default_rng(1).normal(size=(3, H, W)) * keep
    want = ora.render_adjoint(proj, bins, (uC, np.zeros((3, 3, H, W))))["g2d"]
    with gs.Context() as ctx:
        ctx.render_with_grads(gs.DeviceScene(scene), cam, W, H)
        got = ctx.render_backward(_t(uC), None).cpu().numpy()
    bad, worst = _cmp_cols(got, want)
    assert bad == 0, (bad, worst)


# ---------------------------------------------------------------- projection

@pytest.mark.parametrize("sh", [None, 1, 3])
def test_project_backward(gs, ora, sh):
    n, W, H = 2000, 96, 64
    scene = scenes.random_scene(n=n, seed=40 + (sh or 0), sh_degree=sh)
    cam = scenes.pinhole_camera(W, H, viewmat=scenes.look_at_viewmat((0.5, -0.3, -0.4), (0.0, 0.1, 3.0)))
    g2d = np.random.default_rng(2).normal(size=(n, 9)).astype(np.float32)
    want = ora.project_adjoint(scene, cam, W, H, g2d.astype(np.float64))
    with gs.Context() as ctx:
        ctx.project(gs.DeviceScene(scene), cam, W, H)
        got = {k: v.cpu().numpy() for k, v in ctx.project_backward(_t(g2d)).items()}
    # Gaussians whose colour sits at the max(0, .) kink or whose x/z, y/z sits at
    # the frustum clamp take a one-sided derivative that FP32 may pick the other way
    proj = ora.project(scene, cam, W, H)
    pre = np.asarray(proj["rgb"])  # clamped colour; the kink is at 0
    fine = ~np.any(np.abs(pre) < 1e-5, axis=1) | (sh is None)
    for key, w in want.items():
        g = got[key].reshape(n, -1)[fine]
        bad, worst = _cmp_cols(g, w.reshape(n, -1)[fine])
        assert bad == 0, (key, bad, worst)


# ---------------------------------------------------------------- chain

@pytest.mark.parametrize("variant", VARIANTS)
def test_backward_chain_exact(gs, ora, variant):
    """gs_backward (upscale -> blend -> projection adjoints in one call) against
    the oracle's chained adjoints, exact mode (no near-threshold decisions)."""
    n, W, H, s = 300, 40, 32, 2
    scene = scenes.random_scene(n=n, seed=17, sh_degree=2, log_scale_mean=-2.6)
    cam = scenes.pinhole_camera(W, H)
    bg = (0.1, 0.3, 0.2)
    dout = np.random.default_rng(4).normal(size=(3, H * s, W * s)).astype(np.float32)
    proj = ora.project(scene, cam, W, H, mode=1)
    bins = ora.bin_pairs(proj)
    dC, dG = ora.upscale_adjoint(dout.astype(np.float64), W, H)
    g2d = ora.render_adjoint(proj, bins, (dC, dG), bg=bg)["g2d"]
    want = ora.project_adjoint(scene, cam, W, H, g2d)
    with gs.Context(mode="exact", bg=bg, bwd_recompute=variant == "recompute") as ctx:
        ctx.render_with_grads(gs.DeviceScene(scene), cam, W, H)
        got = {k: v.cpu().numpy() for k, v in ctx.backward(_t(dout), s).items()}
        ctx.synchronize()
    for key, w in want.items():
        bad, worst = _cmp_cols(got[key].reshape(n, -1), w.reshape(n, -1), tol_rel=1e-3, tol_abs=1e-3)
        assert bad == 0, (key, bad, worst)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("mode,s", [("3dgs", 2), ("3dgs", 3), ("exact", 2)])
def test_fused_backward_equals_chain(gs, mode, s, variant):
    """gs_backward takes the upscale's adjoint inside the blend's; it equals the
    separate calls (upscale adjoint -> planes -> blend adjoint -> projection
    adjoint) up to the order of the float atomics that sum over tiles."""
    import torch
    n, W, H = 3000, 77, 45
    scene = gs.DeviceScene(scenes.random_scene(n=n, seed=19, sh_degree=3))
    cam = scenes.pinhole_camera(W, H)
    dout = torch.randn(3, H * s, W * s, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    with gs.Context(mode=mode, bg=(0.2, 0.1, 0.4), bwd_recompute=variant == "recompute") as ctx:
        ctx.render_with_grads(scene, cam, W, H)
        fused = {k: v.cpu().numpy() for k, v in ctx.backward(dout, s).items()}
        dC, dG = ctx.upscale_backward(dout, W, H, s)
        g2d = ctx.render_backward(dC, dG)
        chain = {k: v.cpu().numpy() for k, v in ctx.project_backward(g2d).items()}
        ctx.synchronize()
    for k in fused:
        np.testing.assert_allclose(fused[k], chain[k], rtol=1e-5, atol=1e-6 * (np.abs(chain[k]).max() + 1e-12))


def test_autograd_matches_backward(gs):
    """torch.autograd through render_upscale equals gs_backward on the same upstream."""
    import torch
    n, W, H, s = 500, 48, 32, 2
    scene = scenes.random_scene(n=n, seed=23, sh_degree=1)
    cam = scenes.pinhole_camera(W, H)
    params = {k: torch.tensor(np.asarray(scene[k], np.float32), device="cuda", requires_grad=True)
              for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    w = torch.randn(3, H * s, W * s, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    with gs.Context() as ctx:
        out = gs.render_upscale(ctx, cam, W, H, s, params["means"], params["log_scales"], params["quats"],
                                params["opacity_logits"], params["sh"])
        (out * w).sum().backward()
        dev = gs.DeviceScene(scene)
        ctx.render_with_grads(dev, cam, W, H)
        ref = ctx.backward(w.contiguous(), s)
        torch.cuda.synchronize()
    for k, p in params.items():
        np.testing.assert_allclose(p.grad.cpu().numpy(), ref[k].cpu().numpy(), rtol=1e-4,
                                   atol=1e-4 * float(ref[k].abs().max()) + 1e-12)


# ---------------------------------------------------------------- edge cases

def test_backward_not_ready(gs):
    import torch
    W, H = 32, 32
    scene = gs.DeviceScene(scenes.random_scene(n=50, seed=1))
    cam = scenes.pinhole_camera(W, H)
    up = torch.zeros(3, H, W, device="cuda")
    with gs.Context() as ctx:
        with pytest.raises(gs.GSError) as e:
            ctx.n = scene.n
            ctx.render_backward(up)
        assert e.value.status == gs.GS_ERR_NOT_READY
        ctx.render(scene, cam, W, H)                       # plain render: no derivative state
        with pytest.raises(gs.GSError) as e:
            ctx.render_backward(up)
        assert e.value.status == gs.GS_ERR_NOT_READY


def test_backward_empty_and_culled(gs):
    import torch
    W, H, s = 32, 24, 2
    cam = scenes.pinhole_camera(W, H)
    sc = scenes.random_scene(n=20, seed=2)
    sc["means"] = sc["means"].copy()
    sc["means"][:, 2] = -1.0                               # all behind the camera
    with gs.Context() as ctx:
        ctx.render_with_grads(gs.DeviceScene(sc), cam, W, H)
        g = ctx.backward(torch.ones(3, H * s, W * s, device="cuda"), s)
        for v in g.values():
            assert not v.any()
        empty = gs.DeviceScene(scenes.random_scene(n=0, seed=0))
        ctx.render_with_grads(empty, cam, W, H)
        g2 = ctx.render_backward(torch.ones(3, H, W, device="cuda"), torch.ones(3, 3, H, W, device="cuda"))
        assert g2.shape == (0, 9)


# ---------------------------------------------------------------- the two variants

def _opaque_layers(n=6000, seed=61):
    """Stacked high-opacity Gaussians (opacity logits N(3.5, 1): alpha at the
    0.99 clamp or just below it over much of each footprint), so that most
    pixels take several steps of alpha >= 0.9 before they stop: the steps
    whose inversion divides by 1 - alpha <= 0.1."""
    sc = scenes.random_scene(n=n, seed=seed, sh_degree=1, xy_range=0.9, log_scale_mean=-2.9)
    sc["opacity_logits"] = np.random.default_rng(seed).normal(3.5, 1.0, n).astype(np.float32)
    return sc


def _errors(got, want):
    rms = np.sqrt(np.mean(want ** 2, axis=0, keepdims=True)) + 1e-30
    return float(np.max(np.abs(got - want) / (np.abs(want) + rms)))


def test_variants_on_opaque_layers(gs, ora):
    """Both variants against the FP64 adjoint on a scene of opaque layers
    (pixels with several alpha >= 0.9 steps), each within the tolerance; the
    recompute variant's error is at most the inversion's.  Also: the recompute
    variant needs only the projection (no stored forward state)."""
    import torch
    W, H = 96, 64
    scene = _opaque_layers()
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    bins = ora.bin_pairs(proj)
    ref = ora.render(proj, bins, variants=True)
    keep = (ref["nvar"] == 1) & ~borderline_tile_mask(proj)
    assert keep.mean() > 0.8
    rng = np.random.default_rng(8)
    uC = rng.normal(size=(3, H, W)) * keep
    uG = rng.normal(size=(3, 3, H, W)) * keep
    want = ora.render_adjoint(proj, bins, (uC, uG))["g2d"]
    # the scene does what it is for: steps of alpha >= 0.9 are common
    a = np.asarray(proj["opacity"])
    assert np.mean(a > 0.9) > 0.5
    got = {}
    for variant in VARIANTS:
        with gs.Context(bwd_recompute=variant == "recompute") as ctx:
            dev = gs.DeviceScene(scene)
            if variant == "recompute":
                ctx.project(dev, cam, W, H)           # the projection alone suffices
                g = ctx.render_backward(_t(uC), _t(uG))
            else:
                ctx.render_with_grads(dev, cam, W, H)
                g = ctx.render_backward(_t(uC), _t(uG))
            ctx.synchronize()
            got[variant] = g.cpu().numpy()
            torch.cuda.synchronize()
    err = {v: _errors(np.asarray(got[v], np.float64), want) for v in VARIANTS}
    for v in VARIANTS:
        bad, worst = _cmp_cols(got[v], want)
        assert bad == 0, (v, bad, worst, err)
    assert err["recompute"] <= err["inversion"] * 1.05, err


def test_recompute_long_lists_thin_checkpoints(gs, ora):
    """Exact mode, 3000 Gaussians: every tile's list is every Gaussian, so a
    block walks about 12 rounds of 256 candidates, more than the 8 checkpoint
    slots of the recompute variant (which then keeps every second round).
    Both variants against the oracle."""
    W, H = 48, 16
    scene = scenes.random_scene(n=3000, seed=62, log_scale_mean=-2.7)
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H, mode=1)
    bins = ora.bin_pairs(proj)
    rng = np.random.default_rng(9)
    uC = rng.normal(size=(3, H, W))
    uG = rng.normal(size=(3, 3, H, W))
    want = ora.render_adjoint(proj, bins, (uC, uG))["g2d"]
    for variant in VARIANTS:
        with gs.Context(mode="exact", bwd_recompute=variant == "recompute") as ctx:
            ctx.render_with_grads(gs.DeviceScene(scene), cam, W, H)
            got = ctx.render_backward(_t(uC), _t(uG)).cpu().numpy()
            ctx.synchronize()
        bad, worst = _cmp_cols(got, want)
        assert bad == 0, (variant, bad, worst)
