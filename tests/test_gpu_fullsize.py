"""Parity at the full sizes of the scene-shaped workload, run the way the
benchmark runs it.

Workload: 1.5M Gaussians from a seeded 200-component mixture, SH degree 3,
16x16 tiles, 3DGS mode, black background.  Three paths are checked: the
960x540 render with derivatives and its 2x upscale to 1920x1080, the 480x270
render with its 4x upscale, and the direct 1920x1080 render.

Launch configuration: a context for frames without a host wait, with buffers
reserved up front.  Each step is captured once in a CUDA graph and replayed.

The oracle cannot blend a whole frame of this scene in seconds, so it checks
what it can compute one by one:
  - the binning in full: every (tile, depth, id) pair, bit for bit, and the
    per-tile list lengths;
  - a seeded sample of low-res pixels (colour and the three derivative
    planes), plus the last row, the last column and the ragged bottom tile
    row;
  - a seeded sample of upscaled output pixels, computed from the GPU's own C
    and derivative planes, so both sides have identical inputs;
  - the reverse mode for an upstream gradient that is non-zero only on a
    sample of output pixels.  The oracle's adjoints there are exact sums over
    the low-res pixels those outputs read.
Tolerances and exclusions are the ones the small-size parity tests use."""
import numpy as np
import pytest

import scenes
from helpers import (TOL_UP, borderline_pixel_mask, compare_pixels, depth_order_ambiguous, gpu_rows,
                     pairs_without)

pytestmark = pytest.mark.gpu

N = 1_500_000
LOW_W, LOW_H = 960, 540
OUT_W, OUT_H = 1920, 1080


@pytest.fixture(scope="module")
def gs():
    import torch
    import paper_2503_14171_gb300 as gs
    assert torch.cuda.is_available()
    return gs


@pytest.fixture(scope="module")
def scene():
    return scenes.mixture_scene(N, seed=0)


@pytest.fixture(scope="module")
def dev(gs, scene):
    return gs.DeviceScene(scene)


def _graphed(gs, W, H, pairs, body):
    """The benchmark's launch configuration: reserve, run the body once, capture
    it in a CUDA graph, replay it three times.  Returns the open context."""
    import torch
    stream = torch.cuda.Stream()
    ctx = gs.Context(stream=stream, no_host_wait=True)
    ctx.reserve(N, W, H, pairs)
    with torch.cuda.stream(stream):
        body(ctx)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            body(ctx)
        for _ in range(3):
            graph.replay()
    torch.cuda.synchronize()
    ctx.synchronize()                    # raises on a device-side error or overflow
    ctx._graph = graph                   # keep the captured memory alive with the context
    return ctx


def _low_pixels(W, H, m, seed):
    """m seeded pixels, plus the last row and column and the ragged bottom tile row."""
    rng = np.random.default_rng(seed)
    pts = [np.stack([rng.integers(0, W, m), rng.integers(0, H, m)], 1)]
    xs = np.arange(0, W, 7)
    pts.append(np.stack([xs, np.full_like(xs, H - 1)], 1))
    ys = np.arange(0, H, 5)
    pts.append(np.stack([np.full_like(ys, W - 1), ys], 1))
    y0 = (H // 16) * 16
    if y0 < H:
        k = 200
        pts.append(np.stack([rng.integers(0, W, k), rng.integers(y0, H, k)], 1))
    return np.unique(np.concatenate(pts), axis=0).astype(np.int64)


def _high_pixels(W2, H2, m, seed):
    rng = np.random.default_rng(seed)
    pts = [np.stack([rng.integers(0, W2, m), rng.integers(0, H2, m)], 1)]
    for X in (0, W2 - 1):
        ys = np.arange(0, H2, 9)
        pts.append(np.stack([np.full_like(ys, X), ys], 1))
    for Y in (0, H2 - 1):
        xs = np.arange(0, W2, 11)
        pts.append(np.stack([xs, np.full_like(xs, Y)], 1))
    return np.unique(np.concatenate(pts), axis=0).astype(np.int64)


def _check_low(ora, C, G, proj, bins, pix, rotated=False):
    """Sampled pixels against the oracle; excluded: pixels a rect-borderline
    Gaussian can change and, for a rotated camera (FP32 depths not exact),
    pixels whose blend order is not unique."""
    ref = ora.render(proj, bins, pixels=pix, variants=True)
    rows = gpu_rows(C, G, pix) if G is not None else C.cpu().numpy()[:, pix[:, 1], pix[:, 0]].T
    excl = borderline_pixel_mask(proj, pix)
    if rotated:
        excl = excl | depth_order_ambiguous(proj, bins, pix)
    fail, checked, excluded = compare_pixels(rows, ref, exclude=excl)
    assert fail == 0, f"{fail} of {checked} sampled pixels outside tolerance"
    assert checked > 0.9 * len(pix), (checked, excluded)
    return ref


def _borderline_slack(proj):
    """Tiles a rect-borderline Gaussian may or may not cover under FP32
    rounding (its envelope rect minus its core rect), summed."""
    k = 0
    for i in np.nonzero(proj["borderline"])[0]:
        e, c = proj["envelope"][i], proj["core"][i]
        k += max(0, e[2] - e[0] + 1) * max(0, e[3] - e[1] + 1)
        k -= max(0, c[2] - c[0] + 1) * max(0, c[3] - c[1] + 1)
    return int(k)


def _neighbourhood_max(a, r0, r1):
    """max over the window [y + r0, y + r1] x [x + r0, x + r1] (clipped) of a [H, W]."""
    H, W = a.shape
    out = np.full_like(a, -np.inf)
    for dy in range(r0, r1 + 1):
        for dx in range(r0, r1 + 1):
            ys = np.clip(np.arange(H) + dy, 0, H - 1)
            xs = np.clip(np.arange(W) + dx, 0, W - 1)
            out = np.maximum(out, a[ys][:, xs])
    return out


def _check_upscale(ora, C, G, out, pix, W2, H2):
    """Sampled outputs of the upscale against the oracle on the GPU's own
    inputs; the bound scales with the inputs the output pixel reads (its
    4 x 4 low-res neighbourhood, a superset of the cell corners)."""
    Cn = C.cpu().numpy().astype(np.float64)
    Gn = G.cpu().numpy().astype(np.float64)
    H, W = Cn.shape[1:]
    want = ora.upscale(Cn, Gn, W2, H2, pixels=pix)
    got = out.cpu().numpy()[:, pix[:, 1], pix[:, 0]].T
    mag = np.maximum(np.abs(Cn).max(axis=0), np.abs(Gn).reshape(9, H, W).max(axis=0))
    loc = _neighbourhood_max(mag, -1, 2)
    x = np.floor((pix[:, 0] + 0.5) * W / W2 - 0.5).astype(np.int64).clip(0, W - 1)
    y = np.floor((pix[:, 1] + 0.5) * H / H2 - 0.5).astype(np.int64).clip(0, H - 1)
    tol = TOL_UP * (1.0 + loc[y, x])[:, None]
    bad = np.abs(got - want) > tol
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(got - want) / tol)))


# ---------------------------------------------------------------- 960x540 -> 2x

@pytest.fixture(scope="module")
def low(gs, ora, scene, dev):
    import torch
    cam = scenes.pinhole_camera(LOW_W, LOW_H)
    proj = ora.project(scene, cam, LOW_W, LOW_H)
    bins = ora.bin_pairs(proj)
    C = torch.empty(3, LOW_H, LOW_W, device="cuda")
    G = torch.empty(3, 3, LOW_H, LOW_W, device="cuda")
    out = torch.empty(3, OUT_H, OUT_W, device="cuda")

    def body(gc):
        gc.project(dev, cam, LOW_W, LOW_H)
        gc.render_binned(grads=True, out_C=C, out_grads=G)
        gc.upscale(C, G, 2, out=out)

    # super-tile pairs never outnumber tile pairs: the oracle's count with the
    # benchmark's 10 % headroom bounds the reservation
    ctx = _graphed(gs, LOW_W, LOW_H, bins["P"] + bins["P"] // 10 + 4096, body)
    yield dict(ctx=ctx, cam=cam, proj=proj, bins=bins, C=C, G=G, out=out)
    ctx.close()


def test_full_bins(low):
    """Every pair of the 960x540 frame bit for bit (identity-rotation camera:
    the FP32 depth keys are exact), pairs of rect-borderline Gaussians dropped
    on both sides.  The GPU's pairs of those Gaussians lie in their envelope
    rects and cover their core rects; the ranges delimit the GPU's own list."""
    proj, bins, ctx = low["proj"], low["bins"], low["ctx"]
    keys, vals, ranges = (t.cpu().numpy() for t in ctx.read_bins())
    keys, vals, ranges = keys.view(np.uint64), vals.view(np.uint32), ranges.view(np.uint32)
    drop = np.nonzero(proj["borderline"])[0].astype(np.uint32)
    gk, gv = pairs_without(keys, vals, drop)
    rk, rv = pairs_without(bins["keys"], bins["vals"], drop)
    assert len(gk) == len(rk)
    assert np.array_equal(gk, rk)
    assert np.array_equal(gv, rv)

    tiles_x, tiles_y = proj["tiles_x"], proj["tiles_y"]
    T = tiles_x * tiles_y
    t = (keys >> np.uint64(32)).astype(np.int64)
    sel = np.isin(vals, drop)
    bid, bt = vals[sel].astype(np.int64), t[sel]
    env, core = proj["envelope"][bid], proj["core"][bid]
    tx, ty = bt % tiles_x, bt // tiles_x
    assert np.all((tx >= env[:, 0]) & (tx <= env[:, 2]) & (ty >= env[:, 1]) & (ty <= env[:, 3]))
    have = set((bid * T + bt).tolist())
    for i in drop.astype(np.int64):
        c = proj["core"][i]
        for y in range(c[1], c[3] + 1):
            for x in range(c[0], c[2] + 1):
                assert i * T + y * tiles_x + x in have, (i, x, y)

    assert ranges.shape == (T, 2)
    assert np.all(np.diff(t) >= 0)
    s, e = ranges[:, 0].astype(np.int64), ranges[:, 1].astype(np.int64)
    nz = e > s
    assert int((e - s).sum()) == len(keys)
    assert np.all(t[s[nz]] == np.nonzero(nz)[0]) and np.all(t[e[nz] - 1] == np.nonzero(nz)[0])


def test_full_render_sampled(ora, low):
    pix = _low_pixels(LOW_W, LOW_H, 4000, seed=1)
    _check_low(ora, low["C"], low["G"], low["proj"], low["bins"], pix)


def test_full_upscale_2x_sampled(ora, low):
    pix = _high_pixels(OUT_W, OUT_H, 6000, seed=2)
    _check_upscale(ora, low["C"], low["G"], low["out"], pix, OUT_W, OUT_H)


def _check_backward_sampled(ora, scene, n, cam, proj, bins, ctx, upstream, seed):
    """gs_backward for an upstream gradient that is non-zero only on 300
    seeded output pixels (upstream(hx, hy, rng) gives its [3, k] values there),
    against upscale adjoint -> blend adjoint on the low-res pixels they read
    -> projection adjoint of the Gaussians those pixels blend.  Output pixels
    whose cell corners hold a pixel the forward check excludes (near-threshold
    decisions, a rect-borderline Gaussian above the cut-off) are dropped."""
    import torch
    rng = np.random.default_rng(seed)
    hx, hy = rng.integers(0, OUT_W, 300), rng.integers(0, OUT_H, 300)
    # the cell (i, j) = clamp(floor(x), 0, W - 2) of x = (X + 0.5) / 2 - 0.5 and its corners
    cx = np.clip(np.floor((hx + 0.5) / 2 - 0.5).astype(np.int64), 0, LOW_W - 2)
    cy = np.clip(np.floor((hy + 0.5) / 2 - 0.5).astype(np.int64), 0, LOW_H - 2)
    nb = np.array([(dx, dy) for dy in range(2) for dx in range(2)])
    nx = cx[:, None] + nb[None, :, 0]
    ny = cy[:, None] + nb[None, :, 1]
    lp = np.unique(np.stack([nx.ravel(), ny.ravel()], 1), axis=0)
    ref = ora.render(proj, bins, pixels=lp, variants=True)
    bad_lo = np.zeros((LOW_H, LOW_W), bool)
    bad_lo[lp[:, 1], lp[:, 0]] = (ref["nvar"] != 1) | borderline_pixel_mask(proj, lp)
    keep = ~np.any(bad_lo[ny, nx], axis=1)
    assert keep.mean() > 0.7
    dout = np.zeros((3, OUT_H, OUT_W), np.float32)
    dout[:, hy[keep], hx[keep]] = upstream(hx[keep], hy[keep], rng)

    dC, dG = ora.upscale_adjoint(dout.astype(np.float64), LOW_W, LOW_H)
    live = np.any(dC != 0, axis=0) | np.any(dG.reshape(9, LOW_H, LOW_W) != 0, axis=0)
    ly, lx = np.nonzero(live)
    assert not np.any(bad_lo[ly, lx])
    pix = np.stack([lx, ly], 1)
    rows = np.concatenate([dC[:, ly, lx].T, dG.reshape(9, LOW_H, LOW_W)[:, ly, lx].T], axis=1)
    g2d = ora.render_adjoint(proj, bins, rows, pixels=pix)["g2d"]
    hit = np.nonzero(np.any(g2d != 0, axis=1))[0]
    assert len(hit) > 100
    sub = {k: (v[hit] if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    want = ora.project_adjoint(sub, cam, LOW_W, LOW_H, g2d[hit])

    got = ctx.backward(torch.as_tensor(dout).cuda(), 2)
    torch.cuda.synchronize()
    ctx.synchronize()
    got = {k: v.cpu().numpy().reshape(n, -1) for k, v in got.items()}
    # a colour clamped at max(0, .) has a one-sided derivative FP32 may take the other way
    fine = ~np.any(np.abs(proj["rgb"][hit]) < 1e-5, axis=1)
    rest = np.ones(n, bool)
    rest[hit] = False
    for key, w in want.items():
        w = w.reshape(len(hit), -1)
        g = got[key][hit]
        # the derivative tolerance: 1e-3 max(|ref|, rms of the parameter's column)
        rms = np.sqrt(np.mean(w ** 2, axis=0, keepdims=True)) + 1e-30
        tol = 1e-3 * np.maximum(np.abs(w), rms)
        r = np.where(fine[:, None], np.abs(g - w) / tol, 0.0)
        worst = np.unravel_index(np.argmax(r), r.shape)
        assert r.max() <= 1.0, (key, int((r > 1).sum()), float(r.max()), float(w[worst]), float(g[worst]),
                                float(rms[0, worst[1]]))
        # Gaussians no live pixel blends receive nothing
        assert np.all(np.abs(got[key][rest]) <= 5e-4 * rms), key


def test_full_backward_sampled(ora, scene, low):
    """The reverse mode of the 2x step for a seeded normal upstream gradient on
    300 output pixels (the benchmark's scene)."""
    _check_backward_sampled(ora, scene, N, low["cam"], low["proj"], low["bins"], low["ctx"],
                            lambda hx, hy, rng: rng.normal(size=(3, len(hx))).astype(np.float32), seed=5)


def test_differentiation_workload_1m_sampled(gs, ora):
    """The differentiation workload: the mixture scene's generator with 1M
    Gaussians, 960x540 render with derivatives -> 2x upscale -> the loss
    L = 0.8 mean|out - t| + 0.2 mean((out - t)^2) against a seeded target t
    (offset so that no residual sits at the L1 kink), taken over 300 seeded
    output pixels; its upstream gradient (0.8 sign(r) + 0.4 r) / m goes
    through gs_backward in the benchmark's launch configuration and is checked
    against the oracle's adjoint chain as above."""
    import torch
    n = 1_000_000
    scene1 = scenes.mixture_scene(n, seed=0)
    cam = scenes.pinhole_camera(LOW_W, LOW_H)
    proj = ora.project(scene1, cam, LOW_W, LOW_H)
    bins = ora.bin_pairs(proj)
    dev1 = gs.DeviceScene(scene1)
    C = torch.empty(3, LOW_H, LOW_W, device="cuda")
    G = torch.empty(3, 3, LOW_H, LOW_W, device="cuda")
    out = torch.empty(3, OUT_H, OUT_W, device="cuda")

    def body(gc):
        gc.project(dev1, cam, LOW_W, LOW_H)
        gc.render_binned(grads=True, out_C=C, out_grads=G)
        gc.upscale(C, G, 2, out=out)

    stream = torch.cuda.Stream()
    ctx = gs.Context(stream=stream, no_host_wait=True)
    ctx.reserve(n, LOW_W, LOW_H, bins["P"] + bins["P"] // 10 + 4096)
    try:
        with torch.cuda.stream(stream):
            body(ctx)
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                body(ctx)
            graph.replay()
        torch.cuda.synchronize()
        ctx.synchronize()
        o = out.cpu().numpy()
        target = o + 0.05 + 0.1 * np.abs(np.random.default_rng(11).standard_normal(o.shape)).astype(np.float32)

        def upstream(hx, hy, rng):
            r = (o[:, hy, hx] - target[:, hy, hx]).astype(np.float64)
            assert np.all(np.abs(r) > 1e-2)
            m = r.size
            return ((0.8 * np.sign(r) + 0.4 * r) / m).astype(np.float32)

        _check_backward_sampled(ora, scene1, n, cam, proj, bins, ctx, upstream, seed=13)
    finally:
        ctx.close()


# ---------------------------------------------------------------- 480x270 -> 4x

def test_four_x_path_sampled(gs, ora, scene, dev):
    import torch
    W, H = OUT_W // 4, OUT_H // 4
    cam = scenes.pinhole_camera(W, H)
    proj = ora.project(scene, cam, W, H)
    bins = ora.bin_pairs(proj)
    C = torch.empty(3, H, W, device="cuda")
    G = torch.empty(3, 3, H, W, device="cuda")
    out = torch.empty(3, OUT_H, OUT_W, device="cuda")

    def body(gc):
        gc.render_with_grads(dev, cam, W, H, out_C=C, out_grads=G)
        gc.upscale(C, G, 4, out=out)

    ctx = _graphed(gs, W, H, bins["P"] + bins["P"] // 10 + 4096, body)
    try:
        _check_low(ora, C, G, proj, bins, _low_pixels(W, H, 3000, seed=3))
        _check_upscale(ora, C, G, out, _high_pixels(OUT_W, OUT_H, 6000, seed=4), OUT_W, OUT_H)
    finally:
        ctx.close()


# ---------------------------------------------------------------- direct 1920x1080

def test_direct_render_sampled(gs, ora, scene, dev):
    import torch
    cam = scenes.scaled_camera(scenes.pinhole_camera(LOW_W, LOW_H), 2)
    proj = ora.project(scene, cam, OUT_W, OUT_H)
    bins = ora.bin_pairs(proj)
    direct = torch.empty(3, OUT_H, OUT_W, device="cuda")
    ctx = _graphed(gs, OUT_W, OUT_H, bins["P"] + bins["P"] // 10 + 4096,
                   lambda gc: gc.render(dev, cam, OUT_W, OUT_H, out_C=direct))
    try:
        _check_low(ora, direct, None, proj, bins, _low_pixels(OUT_W, OUT_H, 4000, seed=6))
        assert abs(ctx.pair_count() - bins["P"]) <= _borderline_slack(proj)
    finally:
        ctx.close()


# ---------------------------------------------------------------- learned residual, 960x540 -> 4x

def test_full_learned_residual_sampled(gs, ora, low):
    """The fused residual at the size the benchmark measures it (the 960x540
    render of the same frame, 4x to 3840x2160), seeded weights, sampled outputs
    against the spline plus the oracle's residual (kernel precision rules of
    the MLP parity tests)."""
    import torch
    from helpers_mlp import bf16_params, forward_reference, random_theta
    from oracle import mlp
    W2, H2 = LOW_W * 4, LOW_H * 4
    theta = bf16_params(random_theta(np.random.default_rng(11), scale=(0.1, 0.15, 0.2)))
    with gs.Context() as ctx:
        out = ctx.upscale_mlp(low["C"], low["G"], W2, H2, params=torch.as_tensor(theta, dtype=torch.float32).cuda())
        ctx.synchronize()
    pix = _high_pixels(W2, H2, 6000, seed=12)
    Cn = low["C"].cpu().numpy().astype(np.float64)
    Gn = low["G"].cpu().numpy().astype(np.float64)
    ref = forward_reference(theta, mlp.features(Cn, Gn, W2, H2, pix))
    want = ora.upscale(Cn, Gn, W2, H2, pixels=pix) + ref["r"]
    got = out.cpu().numpy()[:, pix[:, 1], pix[:, 0]].T
    H, W = Cn.shape[1:]
    mag = np.maximum(np.abs(Cn).max(axis=0), np.abs(Gn).reshape(9, H, W).max(axis=0))
    loc = _neighbourhood_max(mag, -1, 2)
    x = np.floor((pix[:, 0] + 0.5) * W / W2 - 0.5).astype(np.int64).clip(0, W - 1)
    y = np.floor((pix[:, 1] + 0.5) * H / H2 - 0.5).astype(np.int64).clip(0, H - 1)
    tol = TOL_UP * (1.0 + loc[y, x])[:, None] + ref["e3"]
    keep = ref["keep"]
    assert keep.mean() > 0.9
    bad = (np.abs(got - want) > tol) & keep[:, None]
    assert not bad.any(), (int(bad.sum()), float(np.max(np.abs(got - want)[keep] / tol[keep])))
    assert np.abs(ref["r"]).mean() > 1e-3


# ---------------------------------------------------------------- batched views (16 stereo views, 3 sets)

VIEW_SETS = (300_000, 800_000, 2_000_000)


def test_full_batched_views(gs, ora):
    """The batching workload as the benchmark runs it: 16 stereo views (eyes of
    512x512 to 1104x1032 rendered at half size with derivatives, 2x upscales),
    stereo pair k drawing on Gaussian set k mod 3 of the 300k, 800k and 2M
    mixture scenes, autotuned, captured in a CUDA graph and replayed.  Every
    view equals its single-view render bit for bit, and two views (the
    largest and the smallest) match the oracle on sampled pixels."""
    import torch
    camdefs, eyes = scenes.stereo_views()
    V = len(eyes)
    lows = [(w // 2, h // 2) for w, h in eyes]
    cams = [scenes.pinhole_camera(w, h, viewmat=scenes.look_at_viewmat(e, t)) for (w, h), (e, t) in zip(lows, camdefs)]
    sov = [(v // 2) % len(VIEW_SETS) for v in range(V)]
    sets = [scenes.mixture_scene(n, seed=1) for n in VIEW_SETS]
    devs = [gs.DeviceScene(sc) for sc in sets]
    Wm, Hm = max(w for w, _ in lows), max(h for _, h in lows)
    stream = torch.cuda.Stream()
    ps = 0
    with gs.Context(stream=stream) as probe:
        with torch.cuda.stream(stream):
            for (w, h), cam, k in zip(lows, cams, sov):
                probe.project(devs[k], cam, w, h)
                ps = max(ps, probe.super_pair_count())
    with gs.Context(stream=stream, no_host_wait=True) as ctx:
        ctx.reserve_views(max(VIEW_SETS), V, Wm, Hm, ps + ps // 4 + 4096)
        outs = [[torch.empty(3, h, w, device="cuda"), torch.empty(3, 3, h, w, device="cuda"),
                 torch.empty(3, 2 * h, 2 * w, device="cuda")] for w, h in lows]
        with torch.cuda.stream(stream):
            ctx.render_views(devs, cams, lows, [2] * V, outs=outs, scene_of_view=sov)
            torch.cuda.synchronize()
            ms, best = ctx.autotune_views(devs, cams, lows, [2] * V, outs, reps=2, scene_of_view=sov)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                ctx.render_views(devs, cams, lows, [2] * V, outs=outs, scene_of_view=sov)
            for o in outs:
                for t in o:
                    t.zero_()
            graph.replay()
            graph.replay()
        torch.cuda.synchronize()
        ctx.synchronize()
        got = [[t.cpu().numpy() for t in o] for o in outs]
    with gs.Context() as ref:
        for v, ((w, h), cam) in enumerate(zip(lows, cams)):
            C, G = ref.render_with_grads(devs[sov[v]], cam, w, h)
            up = ref.upscale(C, G, 2).cpu().numpy()
            assert np.array_equal(got[v][0], C.cpu().numpy()), v
            assert np.array_equal(got[v][1], G.cpu().numpy()), v
            assert np.array_equal(got[v][2], up), v
    areas = [w * h for w, h in lows]
    for v in (int(np.argmax(areas)), int(np.argmin(areas))):
        (w, h), cam = lows[v], cams[v]
        proj = ora.project(sets[sov[v]], cam, w, h)
        bins = ora.bin_pairs(proj)
        _check_low(ora, torch.as_tensor(got[v][0]), torch.as_tensor(got[v][1]), proj, bins,
                   _low_pixels(w, h, 2500, seed=20 + v), rotated=True)
    del devs
    torch.cuda.empty_cache()
