"""Batched views (gs_render_views, gs_render_views_scenes): every view of a
batch -- stereo pairs of different sizes, over one Gaussian set or several of
uneven size; one projection launch per set, one depth sort, one emission, one
histogram launch and one launch per pass of the pair sort for all views, one
blend launch and one upscale launch -- equals the single-view render of the
same camera bit for bit, upscales included, in every binning and launch shape;
sampled views of a mixed batch match the oracle; the autotuner picks the
fastest shape; the batch replays from a CUDA graph; and the reservation rules
hold."""
import numpy as np
import pytest

import scenes
from helpers import borderline_tile_mask, compare_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import torch
    import paper_2503_14171_gb300 as gs
    assert torch.cuda.is_available()
    return gs


def stereo_batch(sizes, ipd=0.064, target=(0.0, 0.0, 3.0)):
    """Two cameras (left, right eye) per size, looking at target."""
    cams, szs = [], []
    for k, (W, H) in enumerate(sizes):
        for side in (-0.5, 0.5):
            eye = (side * ipd + 0.05 * k, 0.02 * k, -0.2)
            cams.append(scenes.pinhole_camera(W, H, viewmat=scenes.look_at_viewmat(eye, target)))
            szs.append((W, H))
    return cams, szs


def _single(gs, scene, cam, W, H, bg, factor):
    with gs.Context(bg=bg) as ref:
        C, G = ref.render_with_grads(scene, cam, W, H)
        up = ref.upscale(C, G, factor).cpu().numpy()
        return C.cpu().numpy(), G.cpu().numpy(), up


def _check(gs, scene, cams, szs, factors, outs, bg):
    for v, (cam, (W, H)) in enumerate(zip(cams, szs)):
        C, G, up = _single(gs, scene, cam, W, H, bg, factors[v])
        assert np.array_equal(outs[v][0].cpu().numpy(), C), v
        assert np.array_equal(outs[v][1].cpu().numpy(), G), v
        assert np.array_equal(outs[v][2].cpu().numpy(), up), v


@pytest.mark.parametrize("sh", [3, None])
def test_views_equal_single_view(gs, sh):
    scene = gs.DeviceScene(scenes.random_scene(n=8000, seed=31, sh_degree=sh, xy_range=1.2))
    cams, szs = stereo_batch([(96, 64), (130, 100), (64, 64)])
    factors = [2, 2, 3, 3, 1, 1]
    bg = (0.1, 0.3, 0.5)
    with gs.Context(bg=bg, no_host_wait=True) as ctx:
        ctx.reserve_views(scene.n, len(cams), 130, 100, 400000)
        outs = ctx.render_views(scene, cams, szs, factors)
        ctx.synchronize()
    _check(gs, scene, cams, szs, factors, outs, bg)


@pytest.mark.parametrize("config", range(16))
def test_views_every_launch_shape(gs, config):
    """Each binning and launch shape of the batch (warp map x schedule x
    super-tile side) gives the single-view images bit for bit; twice, so that
    the heaviest-first schedule runs on recorded tile durations."""
    scene = gs.DeviceScene(scenes.random_scene(n=12000, seed=36, sh_degree=2, xy_range=1.3, log_scale_mean=-3.3))
    cams, szs = stereo_batch([(150, 110), (77, 45)])
    factors = [2, 2, 3, 3]
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(scene.n, len(cams), 150, 110, 600000)
        ctx.views_config(config % 2, (config // 2) % 4, 4 if config >= 8 else 0)
        outs = ctx.render_views(scene, cams, szs, factors)
        outs = ctx.render_views(scene, cams, szs, factors, outs=outs)
        ctx.synchronize()
    _check(gs, scene, cams, szs, factors, outs, (0.0, 0.0, 0.0))


def test_views_autotune(gs):
    scene = gs.DeviceScene(scenes.random_scene(n=10000, seed=37, sh_degree=1))
    cams, szs = stereo_batch([(128, 96), (96, 64)])
    factors = [2] * 4
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(scene.n, len(cams), 128, 96, 500000)
        outs = ctx.render_views(scene, cams, szs, factors)
        ms, best = ctx.autotune_views(scene, cams, szs, factors, outs, reps=3)
        assert len(ms) == gs.GS_VIEWS_CONFIGS and all(t > 0 for t in ms)
        assert 0 <= best < gs.GS_VIEWS_CONFIGS and ms[best] == min(ms)
        outs = ctx.render_views(scene, cams, szs, factors, outs=outs)   # with the chosen shape
        ctx.synchronize()
        with pytest.raises(gs.GSError) as e:
            ctx.views_config(2, 0)
        with pytest.raises(gs.GSError):
            ctx.views_config(0, 4)
        assert e.value.status == gs.GS_ERR_INVALID_ARG
        with pytest.raises(gs.GSError) as e:
            ctx.views_config(0, 0, 2)
        assert e.value.status == gs.GS_ERR_INVALID_ARG
    _check(gs, scene, cams, szs, factors, outs, (0.0, 0.0, 0.0))


@pytest.mark.parametrize("schedule", [1, 2, 3])
def test_views_graph_replay(gs, schedule):
    import torch
    scene = gs.DeviceScene(scenes.random_scene(n=6000, seed=32, sh_degree=1))
    cams, szs = stereo_batch([(80, 60), (112, 80)])
    factors = [2] * 4
    stream = torch.cuda.Stream()
    with gs.Context(stream=stream, no_host_wait=True) as ctx:
        ctx.reserve_views(scene.n, 4, 112, 80, 300000)
        ctx.views_config(0, schedule)
        with torch.cuda.stream(stream):
            outs = ctx.render_views(scene, cams, szs, factors)
        torch.cuda.synchronize()
        eager = [[t.cpu().numpy() for t in o] for o in outs]
        for o in outs:
            for t in o:
                t.zero_()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            ctx.render_views(scene, cams, szs, factors, outs=outs)
        graph.replay()
        torch.cuda.synchronize()
        ctx.synchronize()
    for o, e in zip(outs, eager):
        for t, te in zip(o, e):
            assert np.array_equal(t.cpu().numpy(), te)


def test_views_rules(gs):
    scene = gs.DeviceScene(scenes.random_scene(n=500, seed=33))
    cams, szs = stereo_batch([(64, 48)])
    with gs.Context() as ctx:
        with pytest.raises(gs.GSError) as e:
            ctx.render_views(scene, cams, szs)
        assert e.value.status == gs.GS_ERR_NOT_READY
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(500, 2, 64, 48, 10000)
        with pytest.raises(gs.GSError) as e:          # more views than reserved
            c3, s3 = stereo_batch([(64, 48), (32, 32)])
            ctx.render_views(scene, c3, s3)
        assert e.value.status == gs.GS_ERR_CAPACITY
        with pytest.raises(gs.GSError) as e:          # a view larger than reserved
            c2, s2 = stereo_batch([(96, 48)])
            ctx.render_views(scene, c2, s2)
        assert e.value.status == gs.GS_ERR_CAPACITY
        ctx.render_views(scene, cams, szs)
        ctx.synchronize()


def test_views_beyond_persistent_sort(gs):
    """n above the persistent depth sort's capacity (one block per SM, 10240
    Gaussians each): the views take the one-sweep sort path."""
    import torch
    n = 152 * 10240 + 4096
    scene = gs.DeviceScene(scenes.random_scene(n=n, seed=34, log_scale_mean=-4.5))
    cams, szs = stereo_batch([(64, 48)])
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(n, 2, 64, 48, 4 * n)
        outs = ctx.render_views(scene, cams, szs, [2, 2])
        ctx.synchronize()
    _check(gs, scene, cams, szs, [2, 2], outs, (0.0, 0.0, 0.0))
    del outs
    torch.cuda.empty_cache()


def test_views_at_the_view_limit(gs):
    """32 views (the limit: five view bits above the 32 depth bits of the
    batched sort's keys) of a small scene at small and ragged sizes, and a
    single view: each equals its single-view render bit for bit."""
    scene = gs.DeviceScene(scenes.random_scene(n=3000, seed=38, sh_degree=1, xy_range=1.1))
    sizes = [(16 + 3 * k, 12 + 2 * k) for k in range(16)]
    cams, szs = stereo_batch(sizes)
    assert len(cams) == 32
    factors = [1 + (v % 3) for v in range(32)]
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(scene.n, 32, max(w for w, _ in szs), max(h for _, h in szs), 200000)
        outs = ctx.render_views(scene, cams, szs, factors)
        ctx.synchronize()
    _check(gs, scene, cams, szs, factors, outs, (0.0, 0.0, 0.0))
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(scene.n, 1, 64, 48, 200000)
        one = ctx.render_views(scene, cams[:1], [(64, 48)], [2])
        ctx.synchronize()
    _check(gs, scene, cams[:1], [(64, 48)], [2], one, (0.0, 0.0, 0.0))


# ---- batches over several Gaussian sets of uneven size ----------------------

def _mixed_sets():
    """Three Gaussian sets of uneven size and colour model: direct RGB, SH
    degree 1, SH degree 3."""
    return [scenes.random_scene(n=3000, seed=41, xy_range=1.0),
            scenes.random_scene(n=9000, seed=42, sh_degree=1, xy_range=1.2, log_scale_mean=-3.3),
            scenes.random_scene(n=21000, seed=43, sh_degree=3, xy_range=1.3, log_scale_mean=-3.5)]


def translated_stereo(sizes, ipd=0.064):
    """Stereo pairs looking down +z from eyes offset in x and y: identity
    rotations, so every view's FP32 depth keys are exact (the oracle's)."""
    cams, szs = [], []
    for k, (W, H) in enumerate(sizes):
        for side in (-0.5, 0.5):
            vm = np.eye(4, dtype=np.float32)
            vm[0, 3] = -(side * ipd + 0.03 * k)
            vm[1, 3] = -0.02 * k
            cams.append(scenes.pinhole_camera(W, H, viewmat=vm))
            szs.append((W, H))
    return cams, szs


def _mixed_case():
    cams, szs = translated_stereo([(96, 64), (130, 100), (64, 64), (110, 72)])
    scene_of_view = [2, 2, 0, 0, 1, 1, 2, 1]       # uneven: the largest set has three views
    factors = [2, 2, 3, 3, 1, 1, 2, 2]
    return cams, szs, scene_of_view, factors


def _check_mixed(gs, devs, cams, szs, sov, factors, outs, bg):
    for v, (cam, (W, H)) in enumerate(zip(cams, szs)):
        C, G, up = _single(gs, devs[sov[v]], cam, W, H, bg, factors[v])
        assert np.array_equal(outs[v][0].cpu().numpy(), C), v
        assert np.array_equal(outs[v][1].cpu().numpy(), G), v
        assert np.array_equal(outs[v][2].cpu().numpy(), up), v


@pytest.mark.parametrize("config", [0, 3, 5, 8, 14])
def test_mixed_sets_equal_single_views(gs, config):
    """A batch over three Gaussian sets of 3k, 9k and 21k Gaussians: every view
    equals its single-view render bit for bit in several binning and launch
    shapes (twice each, the second on recorded tile durations)."""
    sets = _mixed_sets()
    devs = [gs.DeviceScene(sc) for sc in sets]
    cams, szs, sov, factors = _mixed_case()
    bg = (0.05, 0.1, 0.2)
    with gs.Context(bg=bg, no_host_wait=True) as ctx:
        ctx.reserve_views(max(d.n for d in devs), len(cams), 130, 100, 600000)
        ctx.views_config(config % 2, (config // 2) % 4, 4 if config >= 8 else 0)
        outs = ctx.render_views(devs, cams, szs, factors, scene_of_view=sov)
        outs = ctx.render_views(devs, cams, szs, factors, outs=outs, scene_of_view=sov)
        ctx.synchronize()
        # the batch's pair counts are the sums over its views
        ps, p = ctx.super_pair_count(), ctx.pair_count()
    _check_mixed(gs, devs, cams, szs, sov, factors, outs, bg)
    want_ps = want_p = 0
    for v, (cam, (W, H)) in enumerate(zip(cams, szs)):
        with gs.Context() as ref:
            ref.project(devs[sov[v]], cam, W, H)
            want_ps += ref.super_pair_count()
            want_p += ref.pair_count()
    assert p == want_p
    if config < 8:   # the single-view rule's super-tiles (4 x 4 ones make fewer super-tile pairs)
        assert ps == want_ps
    else:
        assert ps <= want_ps


def test_mixed_sets_match_the_oracle(gs, ora):
    """Two views of a mixed batch, one from the RGB set and one from the SH-3
    set, against the FP64 oracle (tolerances of the parity tests)."""
    sets = _mixed_sets()
    devs = [gs.DeviceScene(sc) for sc in sets]
    cams, szs, sov, factors = _mixed_case()
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(max(d.n for d in devs), len(cams), 130, 100, 600000)
        outs = ctx.render_views(devs, cams, szs, factors, scene_of_view=sov)
        ctx.synchronize()
    for v in (1, 2):
        W, H = szs[v]
        proj = ora.project(sets[sov[v]], cams[v], W, H)
        ref = ora.render(proj, ora.bin_pairs(proj), variants=True)
        fail, checked, excl, worst = compare_render(outs[v][0].cpu().numpy(), outs[v][1].cpu().numpy(), ref,
                                                    exclude=borderline_tile_mask(proj))
        assert fail == 0, (v, fail, checked, worst)
        # the 21k-Gaussian set at 96 x 64 is dense: its rect-borderline
        # Gaussians' tiles (excluded, as in every parity test) cover about 1/6
        assert checked > 0.75 * W * H, (v, checked, excl)


def test_mixed_sets_graph_replay_and_autotune(gs):
    """The autotuner on a mixed batch, then the batch recorded in a CUDA graph
    and replayed on new outputs: equal to the eager batch."""
    import torch
    sets = _mixed_sets()
    devs = [gs.DeviceScene(sc) for sc in sets]
    cams, szs, sov, factors = _mixed_case()
    stream = torch.cuda.Stream()
    with gs.Context(stream=stream, no_host_wait=True) as ctx:
        ctx.reserve_views(max(d.n for d in devs), len(cams), 130, 100, 600000)
        with torch.cuda.stream(stream):
            outs = ctx.render_views(devs, cams, szs, factors, scene_of_view=sov)
            ms, best = ctx.autotune_views(devs, cams, szs, factors, outs, reps=2, scene_of_view=sov)
            assert len(ms) == gs.GS_VIEWS_CONFIGS and ms[best] == min(ms)
            outs = ctx.render_views(devs, cams, szs, factors, outs=outs, scene_of_view=sov)
        torch.cuda.synchronize()
        eager = [[t.cpu().numpy() for t in o] for o in outs]
        for o in outs:
            for t in o:
                t.zero_()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            ctx.render_views(devs, cams, szs, factors, outs=outs, scene_of_view=sov)
        graph.replay()
        torch.cuda.synchronize()
        ctx.synchronize()
    for o, e in zip(outs, eager):
        for t, te in zip(o, e):
            assert np.array_equal(t.cpu().numpy(), te)


def test_mixed_sets_rules(gs):
    sets = _mixed_sets()
    devs = [gs.DeviceScene(sc) for sc in sets]
    cams, szs, sov, factors = _mixed_case()
    with gs.Context(no_host_wait=True) as ctx:
        ctx.reserve_views(devs[1].n, len(cams), 130, 100, 600000)   # smaller than the largest set
        with pytest.raises(gs.GSError) as e:
            ctx.render_views(devs, cams, szs, factors, scene_of_view=sov)
        assert e.value.status == gs.GS_ERR_CAPACITY
        with pytest.raises(gs.GSError) as e:                         # a set index out of range
            ctx.render_views(devs[:2], cams, szs, factors, scene_of_view=[0, 1, 0, 1, 0, 1, 0, 2])
        assert e.value.status == gs.GS_ERR_INVALID_ARG
        ok = [0, 0, 0, 0, 1, 1, 0, 1]
        outs = ctx.render_views(devs[:2], cams, szs, factors, scene_of_view=ok)
        ctx.synchronize()
    _check_mixed(gs, devs, cams, szs, ok, factors, outs, (0.0, 0.0, 0.0))


def test_mixed_sets_with_an_empty_set(gs):
    """A set of no Gaussians beside a non-empty one: its views are background
    only, the others unchanged; and a single view through the several-sets
    call equals its single-view render."""
    empty = gs.DeviceScene(scenes.random_scene(n=0, seed=0))
    full = gs.DeviceScene(scenes.random_scene(n=2500, seed=44, sh_degree=2))
    cams, szs = translated_stereo([(64, 48), (40, 30)])
    sov = [0, 1, 1, 0]
    factors = [2, 2, 3, 3]
    bg = (0.3, 0.2, 0.1)
    with gs.Context(bg=bg, no_host_wait=True) as ctx:
        ctx.reserve_views(full.n, len(cams), 64, 48, 100000)
        outs = ctx.render_views([empty, full], cams, szs, factors, scene_of_view=sov)
        one = ctx.render_views([empty, full], cams[1:2], szs[1:2], [2], scene_of_view=[1])
        ctx.synchronize()
    _check_mixed(gs, [empty, full], cams, szs, sov, factors, outs, bg)
    _check_mixed(gs, [empty, full], cams[1:2], szs[1:2], [1], [2], one, bg)
    for v in (0, 3):
        C = outs[v][0].cpu().numpy()
        assert np.allclose(C, np.array(bg, np.float32)[:, None, None])
        assert not outs[v][1].cpu().numpy().any()
